// dg_residual_static: the residual without any device allocation by the call.
//
// Some applications cannot let a library call cudaMalloc or cudaFree when they evaluate a residual:
// frameworks whose caching allocator has already reserved nearly all device memory (a foreign
// cudaMalloc then fails or fragments their pool), and time-critical loops that cannot accept the
// implicit device synchronisation cudaMalloc/cudaFree may perform. This entry point runs the same
// kernels as dg_residual, but takes its scratch (Gauss values, face traces, gradient and face
// fluxes) from one fixed array that lives in the library's device image.
#include <mutex>

#include "dg_internal.cuh"

namespace dg {

// 16 MiB of FP64 scratch, held by every GPU that loads the library until the process exits.
constexpr long long kStaticScratchDoubles = 2LL << 20;
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double* g_static_ptr[kMaxDevices] = {nullptr};
}  // namespace

// Device address of the scratch array on the current device dev, looked up once per device (the
// array's name in host code is only a host-side stand-in, never a device address). With lazy
// module loading the lookup is what loads the module holding the array and reserves its 16 MiB,
// so dg_mesh_create calls it, and dg_residual_static only reads the address the mesh keeps.
int static_scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(DG_EINVAL, "static scratch: device index out of range");
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    cudaError_t err = cudaGetSymbolAddress(&p, g_static_scratch);
    if (err != cudaSuccess)
      return fail(DG_ECUDA, std::string("dg_residual_static: cudaGetSymbolAddress: ") + cudaGetErrorString(err));
    g_static_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_static_ptr[dev];
  return DG_OK;
}

namespace {
template <int N>
int static_residual(dg_mesh* view, const double* u, double t, double* r, cudaStream_t s) {
  int rc = Driver<N>::gradient(view, u, nullptr, s);
  if (rc) return rc;
  return Driver<N>::residual(view, u, nullptr, t, r, nullptr, false, s);
}
}  // namespace

}  // namespace dg

using namespace dg;

extern "C" int dg_residual_static(dg_mesh* mesh, const double* u, double t, double* r, void* stream) {
  if (!mesh || !u || !r) return fail(DG_EINVAL, "dg_residual_static: null argument");
  const long long E = mesh->E, NP = mesh->np, NF = mesh->nf;
  // single-plane workspace of the residual: U, UF, Q, QF, F_hat
  const long long need = E * (5 * NP + 30 * NF + 15 * NP + 90 * NF + 30 * NF);
  if (need > kStaticScratchDoubles)
    return fail(DG_EINVAL, "dg_residual_static: this mesh needs " + std::to_string(need * 8) +
                               " bytes of scratch; the static scratch holds " +
                               std::to_string(kStaticScratchDoubles * 8) + " bytes (use dg_residual)");
  int dev = 0;
  DG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != mesh->device) return fail(DG_EINVAL, "dg_residual_static: current device is not the mesh's device");
  double* base = mesh->static_scratch;   // looked up by dg_mesh_create on this device
  if (!base) return fail(DG_ECUDA, "dg_residual_static: the mesh holds no scratch address");
  // a view of the mesh that shares its geometry and points its workspace into the static array
  dg_mesh view = *mesh;
  view.prof = Prof();
  view.ws = Workspace();
  view.ws.ug = base;
  view.ws.uf = view.ws.ug + E * 5 * NP;
  view.ws.qg = view.ws.uf + E * 30 * NF;
  view.ws.qf = view.ws.qg + E * 15 * NP;
  view.ws.fh = view.ws.qf + E * 90 * NF;
  cudaStream_t s = (cudaStream_t)stream;
  switch (mesh->n) {
    case 2: return static_residual<2>(&view, u, t, r, s);
    case 3: return static_residual<3>(&view, u, t, r, s);
    case 4: return static_residual<4>(&view, u, t, r, s);
    case 5: return static_residual<5>(&view, u, t, r, s);
    default: return fail(DG_EINVAL, "dg_residual_static: unsupported degree");
  }
}
