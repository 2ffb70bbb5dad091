// Element maps of the two mesh families (Sec. 3.3): box and equiangular cubed-sphere shell.
// The isoparametric geometry of an element is the degree-p interpolant of this map at the GLL
// nodes; the map itself is only evaluated at nodes (and at face corners for connectivity).
#pragma once

#include <math.h>

#include "../../include/dg.h"

namespace dg {

struct MapParams {
  int kind, nx, ny, nz;
  double lx, ly, lz;
  const double* r_layers;  // nz + 1 interfaces (shell)
};

// cube panels: centre direction c, first and second tangential directions a, b (a x b = c)
__host__ __device__ inline void panel_frame(int P, double c[3], double a[3], double b[3]) {
  const double tab[6][9] = {
      {1, 0, 0, 0, 1, 0, 0, 0, 1},  {0, 1, 0, -1, 0, 0, 0, 0, 1}, {-1, 0, 0, 0, -1, 0, 0, 0, 1},
      {0, -1, 0, 1, 0, 0, 0, 0, 1}, {0, 0, 1, 0, 1, 0, -1, 0, 0}, {0, 0, -1, 0, 1, 0, 1, 0, 0}};
  for (int d = 0; d < 3; ++d) {
    c[d] = tab[P][d];
    a[d] = tab[P][3 + d];
    b[d] = tab[P][6 + d];
  }
}

// position of reference point (x1, x2, x3) in [-1,1]^3 of element e
__host__ __device__ inline void map_point(const MapParams& mp, long long e, double x1, double x2,
                                          double x3, double out[3]) {
  double s1 = 0.5 * (1.0 + x1), s2 = 0.5 * (1.0 + x2), s3 = 0.5 * (1.0 + x3);
  if (mp.kind == DG_KIND_BOX) {
    long long i = e % mp.nx;
    long long j = (e / mp.nx) % mp.ny;
    long long k = e / ((long long)mp.nx * mp.ny);
    out[0] = (i + s1) * (mp.lx / mp.nx);
    out[1] = (j + s2) * (mp.ly / mp.ny);
    out[2] = (k + s3) * (mp.lz / mp.nz);
    return;
  }
  long long k = e % mp.nz;
  long long rest = e / mp.nz;
  long long i = rest % mp.nx;
  long long j = (rest / mp.nx) % mp.nx;
  int P = (int)(rest / ((long long)mp.nx * mp.nx));
  double dang = 0.5 * M_PI / mp.nx;
  double alpha = -0.25 * M_PI + (i + s1) * dang;
  double beta = -0.25 * M_PI + (j + s2) * dang;
  double c[3], a[3], b[3];
  panel_frame(P, c, a, b);
  double ta = tan(alpha), tb = tan(beta);
  double dir[3], nrm = 0.0;
  for (int d = 0; d < 3; ++d) {
    dir[d] = c[d] + ta * a[d] + tb * b[d];
    nrm += dir[d] * dir[d];
  }
  nrm = sqrt(nrm);
  double r = mp.r_layers[k] + s3 * (mp.r_layers[k + 1] - mp.r_layers[k]);
  for (int d = 0; d < 3; ++d) out[d] = r * dir[d] / nrm;
}

}  // namespace dg
