// Nodal -> Gauss values and face traces (the k_interp step) on the 5th-generation tensor cores, to
// FP64 accuracy.
//
// The step is one dense contraction per element: with A the (N^3 + 6 N^2) x N^3 operator that maps
// the GLL nodal values of one variable to its Gauss values (B x B x B) and to its six face traces
// (the Gauss values extrapolated with e_L / e_R along the face normal), the outputs of all
// variables of a group of elements are A X, X holding one column per (element, variable).
//
// FP64 on FP16 tensor cores by error-free slicing (Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix multiplication and
// its applications", 2012; done here with integer digits):
//   * each operator row is scaled by a power of two 2^(53 - f_r) with |A_rk| < 2^f_r and rounded
//     to an integer, each data column likewise with its largest exponent e_c (exact for the
//     column's largest values); both integers are at most 2^53 and are written as seven balanced
//     digits, six of base 256 (each in [-128, 128]) under a leading one of at most 33, all exact in
//     FP16: A_rk 2^(53 - f_r) = sum_j a_j 2^(8 (6 - j)), X_kc 2^(53 - e_c) = sum_i x_i 2^(8 (6 - i));
//   * the digit products of level l = i + j <= 7 are accumulated by tcgen05.mma (kind::f16, FP32
//     accumulators in tensor memory), one accumulator per level: every term is an integer of at
//     most 2^14 and a level sums at most 7 x 125 of them, below 2^24, so FP32 holds each level
//     exactly;
//   * the levels are combined in 64-bit integers, T = sum_{l<=5} acc_l 2^(8 (5 - l)) +
//     round((2^8 acc_6 + acc_7) / 2^16), and T 2^(f_r + e_c - 50) is rounded once to FP64 from its
//     bits.
// The dropped levels l >= 8 and the roundings of the operands leave an error of about 1e-15 of the
// column's largest value (the sum-factorised FP64 passes: about 2e-16).

//
// Data movement: the operator's digit slices are laid out on the host in the MMA's shared-memory
// operand layout (K-major, no swizzle: 8-row x 16-byte core matrices) and streamed into shared
// memory with bulk copies (cp.async.bulk) through a two-slot ring; the data columns are split into
// digits by the CUDA cores straight into the same layout; the accumulators are read back with
// tcgen05.ld. One persistent CTA per SM (the digits of 64 columns and the ring take 180 KB; the
// eight level accumulators of 64 columns fill the 512 columns of tensor memory).
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dg_internal.cuh"

namespace dg {
namespace {

constexpr int TC_L = 7;          // digits per operand
constexpr int TC_LV = 8;         // digit-product levels kept (l = i + j <= 7)
constexpr int TC_NT = 64;        // data columns per group (MMA N)
constexpr int TC_M = 128;        // operator rows per tile (MMA M)
constexpr int TC_THREADS = 512;
constexpr int TC_TMEM_COLS = 512;
constexpr unsigned TC_WAIT_LIMIT = 1u << 24;   // bounded mbarrier waits (the kernel then reports)

template <int N>
struct TcShape {
  static constexpr int NP = N * N * N, NF = N * N;
  static constexpr int KT = (NP + 15) / 16 * 16;      // K padded to the MMA's K step of 16
  static constexpr int KC = KT / 8;                    // 16-byte chunks per operand row
  static constexpr int ROWS = NP + 6 * NF;
  static constexpr int MT = (ROWS + TC_M - 1) / TC_M;
  static constexpr int ASLICE = TC_M * KT * 2;         // bytes of one operator digit slice of one tile
  static constexpr int XSLICE = TC_NT * KT * 2;        // bytes of one data digit slice
  static constexpr size_t SMEM = (size_t)TC_L * XSLICE + 2 * (size_t)ASLICE + TC_NT * sizeof(int);
};

// byte offset of (row, k) in a K-major, non-swizzled operand of KC 16-byte chunks per row
__host__ __device__ inline int operand_offset(int row, int k, int kc_per_row) {
  return (row >> 3) * (kc_per_row * 128) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// ---------------------------------------------------------------------------------------------
// PTX wrappers (tcgen05, mbarrier, bulk copy)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t operand_desc(uint32_t addr, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;   // leading byte offset: next core matrix along K
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;    // stride byte offset: next group of 8 rows
  d |= (uint64_t)1 << 46;                          // descriptor version of this architecture
  return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// waits for the phase of the given parity to complete; false after TC_WAIT_LIMIT attempts
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned it = 0; it < TC_WAIT_LIMIT; ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}

// ---------------------------------------------------------------------------------------------
// digits and their recombination
// ---------------------------------------------------------------------------------------------
// The seven balanced digits of round(x 2^(53 - e)), e = eb_max - 1022 the exponent bound of the
// column (eb_max its largest biased exponent): d[0] most significant. Zeros and subnormals give
// zero digits (they lie below 2^-1022, far under the column's last digit).
__device__ __forceinline__ void digits_of(double x, int eb_max, int (&d)[TC_L]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)((b >> 52) & 0x7FF);
  const int s = eb_max - eb;       // >= 0: the 53-bit mantissa shifted right by s, rounded
  long long X = 0;
  if (eb != 0 && s < 54) {
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    X = (long long)(s == 0 ? m : (m + (1ull << (s - 1))) >> s);
    if (b >> 63) X = -X;
  }
#pragma unroll
  for (int i = TC_L - 1; i > 0; --i) {
    const int lo = (int)((unsigned)(unsigned long long)X << 24) >> 24;   // low byte, sign-extended
    d[i] = lo;
    X = (X - lo) >> 8;
  }
  d[0] = (int)X;
}

// two digits as the bits of an FP16 pair: 1536 + d is exact in FP16 for |d| < 512 and its bits are
// 0x6600 + d, so subtracting 1536 leaves d exactly
__device__ __forceinline__ uint32_t half2_of(int a, int b) {
  const uint32_t w = __byte_perm((uint32_t)(0x6600 + a), (uint32_t)(0x6600 + b), 0x5410);
  __half2 h = *reinterpret_cast<const __half2*>(&w);
  h = __hsub2(h, __halves2half2(__ushort_as_half(0x6600), __ushort_as_half(0x6600)));
  return *reinterpret_cast<const uint32_t*>(&h);
}

// T 2^k rounded to the nearest FP64 (ties to even), from the bits of T
__device__ __forceinline__ double scaled_double(long long T, int k) {
  if (T == 0) return 0.0;
  const unsigned long long sign = T < 0 ? (1ull << 63) : 0ull;
  unsigned long long a = T < 0 ? (unsigned long long)(-T) : (unsigned long long)T;
  const int lz = __clzll((long long)a);
  a <<= lz;                                   // bit 63 set: T = a 2^-lz
  unsigned long long m = a >> 11;             // 53 leading bits
  const unsigned rem = (unsigned)(a & 0x7FF);
  m += (rem > 0x400u || (rem == 0x400u && (m & 1ull))) ? 1ull : 0ull;
  int eb = 63 - lz + k + 1023;                // biased exponent of (m / 2^52) 2^(63 - lz + k)
  if (m >> 53) {
    m >>= 1;
    ++eb;
  }
  if (eb <= 0 || eb >= 2047) return scalbn((double)T, k);   // outside the normal range
  return __longlong_as_double((long long)(sign | ((unsigned long long)eb << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

// ---------------------------------------------------------------------------------------------
// the kernel
// ---------------------------------------------------------------------------------------------
// u (and v for NC = 2): [E][5][NP] nodal values; outputs as k_interp: ug[pl][E][5][NP] and
// uf[pl][E][6][5][NF], planes plane_g / plane_f apart. aslices: [MT][TC_L] operator digit slices in
// the operand layout; rowexp: [MT * 128] row exponents f_r.
template <int N, int NC>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_interp_tc(const double* __restrict__ u, const double* __restrict__ v, long long E,
                const unsigned char* __restrict__ aslices, const int* __restrict__ rowexp, double* __restrict__ ug,
                double* __restrict__ uf, long long plane_g, long long plane_f, int* __restrict__ err) {
  using S = TcShape<N>;
  constexpr int NP = S::NP, NF = S::NF, KT = S::KT, KC = S::KC, MT = S::MT, ROWS = S::ROWS;
  constexpr int C = 5 * NC, EPG = TC_NT / C, KSTEPS = KT / 16;
  constexpr uint32_t SBO_A = KC * 128, SBO_X = KC * 128;
  constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(TC_NT >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* xs = smem;                                  // [TC_L][XSLICE] data digits
  unsigned char* as = smem + (size_t)TC_L * S::XSLICE;       // [2][ASLICE] operator digit ring
  int* colexp = reinterpret_cast<int*>(as + 2 * (size_t)S::ASLICE);   // [TC_NT] largest biased exponent
  __shared__ __align__(8) uint64_t bar_full[2], bar_empty[2], bar_mma;
  __shared__ uint32_t tmem_holder;
  __shared__ int abort_flag;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_holder)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t == 0) {
    mbar_init(smem_addr(&bar_full[0]), 1);
    mbar_init(smem_addr(&bar_full[1]), 1);
    mbar_init(smem_addr(&bar_empty[0]), 1);
    mbar_init(smem_addr(&bar_empty[1]), 1);
    mbar_init(smem_addr(&bar_mma), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_holder;

  const long long ngroups = (E + EPG - 1) / EPG;
  const long long my_groups = blockIdx.x < ngroups ? (ngroups - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const long long n_slices = my_groups * MT * TC_L;   // operator slices this CTA streams
  // producer state (thread 0): slices q < loaded have been requested
  long long loaded = 0;
  auto issue_load = [&](long long q) {
    const int b = (int)(q & 1);
    const int sl = (int)(q % (MT * TC_L));            // (tile, digit) of stream position q
    bulk_load(smem_addr(as + (size_t)b * S::ASLICE), aslices + (size_t)sl * S::ASLICE, S::ASLICE,
              smem_addr(&bar_full[b]));
  };
  if (t == 0) {
    for (; loaded < 2 && loaded < n_slices; ++loaded) issue_load(loaded);
  }
  bool ok = true;          // this thread's waits all completed
  long long q = 0;         // stream position of the next slice to consume
  long long landed = 0;    // thread 0: slices whose bulk copy it has seen complete (in order)
  uint32_t mma_phase = 0;

  for (long long grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
    const long long e0 = grp * EPG;
    // 1. largest exponent of every data column (a column's KC chunks sit in KC adjacent lanes)
    for (int it = t; it < TC_NT * KC; it += TC_THREADS) {
      const int n = it / KC, kc = it % KC;
      const int el = n / C, cc = n % C;
      const long long e = e0 + el;
      int emax = 0;
      if (el < EPG && e < E) {
        const double* src = (cc < 5 ? u : v) + (e * 5 + cc % 5) * NP;
#pragma unroll
        for (int k8 = 0; k8 < 8; ++k8) {
          const int k = kc * 8 + k8;
          if (k < NP) emax = max(emax, (int)((__double_as_longlong(src[k]) >> 52) & 0x7FF));
        }
      }
#pragma unroll
      for (int off = KC / 2; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
      if (kc == 0) colexp[n] = emax;
    }
    __syncthreads();
    // 2. digits of every data value, 8 consecutive k per thread, into the TC_L slices (lanes take
    //    consecutive columns of one 8-row group: each 16-byte store phase covers 128 contiguous bytes)
    for (int it = t; it < TC_NT * KC; it += TC_THREADS) {
      const int n = (it / (8 * KC)) * 8 + (it & 7), kc = (it >> 3) % KC;
      const int el = n / C, cc = n % C;
      const long long e = e0 + el;
      const int emax = colexp[n];
      int d[8][TC_L];
      const double* src = (cc < 5 ? u : v) + (e * 5 + cc % 5) * NP;
      const bool col_ok = el < EPG && e < E && emax != 2047;
#pragma unroll
      for (int k8 = 0; k8 < 8; ++k8) {
        const int k = kc * 8 + k8;
        const double x = (col_ok && k < NP) ? src[k] : 0.0;
        digits_of(x, emax, d[k8]);
      }
      const int off = operand_offset(n, kc * 8, KC);
#pragma unroll
      for (int i = 0; i < TC_L; ++i) {
        uint4 w;
        w.x = half2_of(d[0][i], d[1][i]);
        w.y = half2_of(d[2][i], d[3][i]);
        w.z = half2_of(d[4][i], d[5][i]);
        w.w = half2_of(d[6][i], d[7][i]);
        *reinterpret_cast<uint4*>(xs + (size_t)i * S::XSLICE + off) = w;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> MMA reads
    __syncthreads();

    for (int mt = 0; mt < MT; ++mt) {
      // 3. one elected thread issues the level products of this tile
      if (t == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int j = 0; j < TC_L; ++j, ++q) {
          const int b = (int)(q & 1);
          if (ok) ok = mbar_wait(smem_addr(&bar_full[b]), (uint32_t)((q >> 1) & 1));
          if (ok) ++landed;
          if (ok) {
            const uint32_t abase = smem_addr(as + (size_t)b * S::ASLICE);
            for (int i = 0; i < TC_L && i + j < TC_LV; ++i) {
              const int lvl = i + j;
              const uint32_t xbase = smem_addr(xs + (size_t)i * S::XSLICE);
              const uint32_t dt = tmem + (uint32_t)(lvl * TC_NT);
              const bool first = j == (lvl >= TC_L ? lvl - (TC_L - 1) : 0);   // first product of the level
#pragma unroll
              for (int ks = 0; ks < KSTEPS; ++ks)
                mma_f16(dt, operand_desc(abase + ks * 256, SBO_A), operand_desc(xbase + ks * 256, SBO_X), IDESC,
                        (!first || ks > 0) ? 1u : 0u);
            }
          }
          mma_commit(smem_addr(&bar_empty[b]));
          // refill the slot of the previous slice once its products are done
          if (q >= 1 && loaded < n_slices) {
            const long long pq = q - 1;
            if (ok) ok = mbar_wait(smem_addr(&bar_empty[pq & 1]), (uint32_t)((pq >> 1) & 1));
            if (ok) issue_load(loaded++);
          }
        }
        mma_commit(smem_addr(&bar_mma));
      } else {
        q += TC_L;
      }
      // 4. every thread: its accumulator row, the levels combined and scaled
      if (ok) ok = mbar_wait(smem_addr(&bar_mma), mma_phase);
      mma_phase ^= 1u;
      if (!ok) atomicOr(&abort_flag, 1);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      {
        constexpr int SEG = TC_NT / 4;                    // columns per warp
        const int quarter = warp & 3, seg = warp >> 2;   // TMEM lanes 32 quarter ..; columns SEG seg ..
        const int r = mt * TC_M + quarter * 32 + lane;
        const bool row_ok = r < ROWS;
        const int fr = row_ok ? rowexp[r] : 0;
        const bool bad = !ok || abort_flag != 0;
        long long obase, ostride_e, ostride_c, oplane;     // output offset of (plane, element, variable)
        double* out;
        if (r < NP) {
          out = ug;
          obase = r;
          ostride_e = 5 * NP;
          ostride_c = NP;
          oplane = plane_g;
        } else {
          const int rr = r - NP, phi = rr / NF, f = rr % NF;
          out = uf;
          obase = (long long)phi * 5 * NF + f;
          ostride_e = 30 * NF;
          ostride_c = NF;
          oplane = plane_f;
        }
#pragma unroll 1
        for (int c4 = 0; c4 < SEG / 4; ++c4) {
          const int col0 = seg * SEG + c4 * 4;
          uint32_t lv[TC_LV][4];
#pragma unroll
          for (int l = 0; l < TC_LV; ++l)
            tmem_ld4(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(l * TC_NT + col0), lv[l]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int ci = 0; ci < 4; ++ci) {
            const int n = col0 + ci;
            const int el = n / C, cc = n % C;
            const long long e = e0 + el;
            if (!row_ok || el >= EPG || e >= E) continue;
            const int emax = colexp[n];
            double val;
            if (bad || emax == 2047) {
              val = __longlong_as_double(0x7FF8000000000000ll);   // NaN in, or the wait gave up
            } else {
              long long T = __float2int_rn(__uint_as_float(lv[0][ci]));
#pragma unroll
              for (int l = 1; l < TC_LV - 2; ++l) T = T * 256 + __float2int_rn(__uint_as_float(lv[l][ci]));
              const long long tail = (long long)__float2int_rn(__uint_as_float(lv[TC_LV - 2][ci])) * 256 +
                                     __float2int_rn(__uint_as_float(lv[TC_LV - 1][ci]));
              T += (tail + 32768) >> 16;
              val = scaled_double(T, fr + (emax - 1022) - 50);
            }
            out[(cc / 5) * oplane + e * ostride_e + (cc % 5) * ostride_c + obase] = val;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();   // the accumulators are free for the next tile
    }
  }
  if (!ok) atomicOr(err, 1);
  // every bulk copy this CTA issued lands before it exits (after a failed wait, the ones not seen
  // complete are waited for here, each wait bounded)
  if (t == 0) {
    for (long long pq = landed; pq < loaded; ++pq)
      if (!mbar_wait(smem_addr(&bar_full[pq & 1]), (uint32_t)((pq >> 1) & 1))) atomicOr(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
  }
}

// ---------------------------------------------------------------------------------------------
// host: the operator's digit slices
// ---------------------------------------------------------------------------------------------
uint16_t fp16_bits_of_small_int(int d) {   // |d| <= 2048: exact in FP16
  if (d == 0) return 0;
  const uint16_t sign = d < 0 ? 0x8000 : 0;
  unsigned a = (unsigned)(d < 0 ? -d : d);
  int e = 31 - __builtin_clz(a);           // 2^e <= a < 2^(e+1)
  const unsigned mant = (a << (10 - e)) & 0x3FF;
  return (uint16_t)(sign | ((unsigned)(e + 15) << 10) | mant);
}

template <int N>
int build_operator(dg_mesh* m) {
  using S = TcShape<N>;
  constexpr int NP = S::NP, NF = S::NF, KT = S::KT, MT = S::MT, ROWS = S::ROWS;
  const Ops& o = m->ops;
  // rows: Gauss values (B x B x B), then face traces phi * NF + f (e_L / e_R along the normal)
  std::vector<long double> A((size_t)MT * TC_M * KT, 0.0L);
  for (int g = 0; g < NP; ++g) {
    const int g0 = g % N, g1 = (g / N) % N, g2 = g / (N * N);
    for (int k = 0; k < NP; ++k) {
      const int k0 = k % N, k1 = (k / N) % N, k2 = k / (N * N);
      A[(size_t)g * KT + k] = (long double)o.B[g0 * N + k0] * o.B[g1 * N + k1] * o.B[g2 * N + k2];
    }
  }
  for (int phi = 0; phi < 6; ++phi) {
    const int axis = phi >> 1;
    const double* ev = (phi & 1) ? o.eR : o.eL;
    for (int f = 0; f < NF; ++f) {
      const int is = f % N, it = f / N;
      for (int j = 0; j < N; ++j) {
        const int i0 = axis == 0 ? j : is, i1 = axis == 0 ? is : (axis == 1 ? j : it), i2 = axis == 2 ? j : it;
        const int g = i0 + N * (i1 + N * i2);
        for (int k = 0; k < NP; ++k) A[(size_t)(NP + phi * NF + f) * KT + k] += (long double)ev[j] * A[(size_t)g * KT + k];
      }
    }
  }
  std::vector<int> rowexp((size_t)MT * TC_M, 0);
  std::vector<uint16_t> sl((size_t)MT * TC_L * TC_M * KT, 0);
  for (int r = 0; r < ROWS; ++r) {
    int fr = INT_MIN;
    for (int k = 0; k < NP; ++k) {
      const double a = (double)A[(size_t)r * KT + k];
      if (a != 0.0) {
        int e;
        std::frexp(a, &e);   // |a| < 2^e
        fr = std::max(fr, e);
      }
    }
    if (fr == INT_MIN) fr = 0;
    rowexp[r] = fr;
    const int mt = r / TC_M, rl = r % TC_M;
    for (int k = 0; k < NP; ++k) {
      long long X = std::llrint(std::ldexp((double)A[(size_t)r * KT + k], 53 - fr));
      int d[TC_L];
      for (int i = TC_L - 1; i > 0; --i) {
        long long lo = X & 0xFF;
        if (lo >= 128) lo -= 256;
        d[i] = (int)lo;
        X = (X - lo) / 256;
      }
      d[0] = (int)X;
      for (int j = 0; j < TC_L; ++j) {
        const size_t base = ((size_t)mt * TC_L + j) * (S::ASLICE / 2);
        sl[base + operand_offset(rl, k, S::KC) / 2] = fp16_bits_of_small_int(d[j]);
      }
    }
  }
  DG_CUDA_TRY(cudaMalloc(&m->tc_aslices, sl.size() * sizeof(uint16_t)));
  DG_CUDA_TRY(cudaMalloc(&m->tc_rowexp, rowexp.size() * sizeof(int)));
  DG_CUDA_TRY(cudaMalloc(&m->tc_err, sizeof(int)));
  DG_CUDA_TRY(cudaMemcpy(m->tc_aslices, sl.data(), sl.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemcpy(m->tc_rowexp, rowexp.data(), rowexp.size() * sizeof(int), cudaMemcpyHostToDevice));
  DG_CUDA_TRY(cudaMemset(m->tc_err, 0, sizeof(int)));
  return DG_OK;
}

}  // namespace

template <int N, int NC>
int interp_tc(dg_mesh* m, const double* u, const double* v, double* ug, double* uf, cudaStream_t s) {
  using S = TcShape<N>;
  if (!m->tc_aslices) return fail(DG_EINVAL, "k_interp_tc: operator not prepared (dg_mesh_set_interp)");
  constexpr int EPG = TC_NT / (5 * NC);
  const long long ngroups = (m->E + EPG - 1) / EPG;
  int sms = 0;
  DG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
  const unsigned grid = (unsigned)std::min<long long>(ngroups, sms);
  auto kern = k_interp_tc<N, NC>;
  DG_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM));
  prof_begin(m, s, KK_INTERP);
  kern<<<grid, TC_THREADS, S::SMEM, s>>>(u, v, m->E, reinterpret_cast<const unsigned char*>(m->tc_aslices),
                                         m->tc_rowexp, ug, uf, m->E * 5 * S::NP, m->E * 30 * S::NF, m->tc_err);
  prof_end(m, s);
  DG_LAUNCH_CHECK("k_interp_tc");
  return DG_OK;
}

template int interp_tc<2, 1>(dg_mesh*, const double*, const double*, double*, double*, cudaStream_t);
template int interp_tc<2, 2>(dg_mesh*, const double*, const double*, double*, double*, cudaStream_t);
template int interp_tc<3, 1>(dg_mesh*, const double*, const double*, double*, double*, cudaStream_t);
template int interp_tc<3, 2>(dg_mesh*, const double*, const double*, double*, double*, cudaStream_t);
template int interp_tc<4, 1>(dg_mesh*, const double*, const double*, double*, double*, cudaStream_t);
template int interp_tc<4, 2>(dg_mesh*, const double*, const double*, double*, double*, cudaStream_t);
template int interp_tc<5, 1>(dg_mesh*, const double*, const double*, double*, double*, cudaStream_t);
template int interp_tc<5, 2>(dg_mesh*, const double*, const double*, double*, double*, cudaStream_t);

int interp_tc_prepare(dg_mesh* m) {
  if (m->tc_aslices) return DG_OK;
  switch (m->n) {
    case 2: return build_operator<2>(m);
    case 3: return build_operator<3>(m);
    case 4: return build_operator<4>(m);
    case 5: return build_operator<5>(m);
    default: return fail(DG_EINVAL, "k_interp_tc: unsupported degree");
  }
}

void interp_tc_release(dg_mesh* m) {
  cudaFree(m->tc_aslices);
  cudaFree(m->tc_rowexp);
  cudaFree(m->tc_err);
  m->tc_aslices = nullptr;
  m->tc_rowexp = nullptr;
  m->tc_err = nullptr;
}

}  // namespace dg
