// Bulk-copy-fed CSR SpMV for the large level operators (K0, K1, their FP64
// residuals).  Rows are cut at setup into tiles of at most kTileNnz stored
// entries and kTileRows rows.  One producer thread moves each tile's values,
// column indices and row pointers (three contiguous ranges, widened to
// 16-byte boundaries) into a 3-stage shared-memory ring with cp.async.bulk
// (evict-first in L2); four consumer warps then compute one row per lane
// from shared memory, gathering x from L2.  A row's sum runs sequentially in
// one thread: no shuffle trees, so FP64 products cost one DFMA each (GB300's
// FP64 rate is low) and FP32 lanes stay busy.
#include <algorithm>

#include "common.cuh"
#include "tma.cuh"

namespace sd {

constexpr int kSpNCW = 4;

template <typename TA>
struct SpTile {
  static constexpr int VA = 16 / sizeof(TA);  // value entries per 16 bytes
};

template <typename TA, typename TX, typename TB, typename TY, typename TACC, int MODE>
__global__ void __launch_bounds__(32 * (kSpNCW + 1), 4) k_spmv_tma(
    int ntiles, const int* __restrict__ trow, const int* __restrict__ rowptr, const int* __restrict__ col,
    const TA* __restrict__ val, const TX* __restrict__ x, const TB* __restrict__ b, TY* __restrict__ y, double s0,
    double s1, const uint8_t* __restrict__ kind, int val_bytes, int col_bytes, int rp_bytes, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int STAGES = 3;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + STAGES;
  const int stage_bytes = val_bytes + col_bytes + rp_bytes;
  unsigned char* stage0 = smem + 128;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, kSpNCW);
    }
    *reinterpret_cast<volatile int*>(empty + STAGES) = 0;  // consumer abort flag
    mbar_fence_init();
  }
  __syncthreads();
  constexpr int VA = 16 / (int)sizeof(TA);
  if (warp == kSpNCW) {
    if (lane == 0) {
      const uint64_t pol = policy_evict_first();
      int k = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = k % STAGES;
        if (k >= STAGES && !mbar_wait(empty + s, ((k / STAGES) - 1) & 1)) {
          atomicOr(err, 1);
          break;
        }
        const int r0 = trow[t], r1 = trow[t + 1];
        const int n0 = rowptr[r0], n1 = rowptr[r1];
        const int va0 = n0 / VA * VA, va1 = (n1 + VA - 1) / VA * VA;
        const int c0 = n0 / 4 * 4, c1 = (n1 + 3) / 4 * 4;
        const int p0 = r0 / 4 * 4, p1 = (r1 + 1 + 3) / 4 * 4;
        const uint32_t vb = (uint32_t)(va1 - va0) * sizeof(TA), cb = (uint32_t)(c1 - c0) * 4u,
                       pb = (uint32_t)(p1 - p0) * 4u;
        unsigned char* st = stage0 + (size_t)s * stage_bytes;
        // a tile of empty rows (e.g. Dirichlet rows of P) has no values or
        // columns to move: only nonzero-size copies are issued
        mbar_expect_tx(full + s, vb + cb + pb);
        if (vb) bulk_g2s(st, val + va0, vb, full + s, pol);
        if (cb) bulk_g2s(st + val_bytes, col + c0, cb, full + s, pol);
        bulk_g2s(st + val_bytes + col_bytes, rowptr + p0, pb, full + s, pol);
      }
      for (int kk = max(0, k - STAGES); kk < k; ++kk)
        if (!mbar_wait(full + (kk % STAGES), (kk / STAGES) & 1)) atomicOr(err, 4);
    }
    return;
  }
  const int ct = threadIdx.x;  // consumer thread 0 .. 32*kSpNCW-1
  constexpr int NC = 32 * kSpNCW;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + STAGES);
  int k = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
    const int s = k % STAGES;
    // the consumer warps agree on a timed-out wait and leave together, so no
    // warp is left waiting at the named barrier
    if (!mbar_wait(full + s, (k / STAGES) & 1)) {
      atomicOr(err, 2);
      *abort_flag = 1;
    }
    asm volatile("bar.sync 1, %0;" ::"r"(NC) : "memory");
    if (*abort_flag) return;
    unsigned char* st = stage0 + (size_t)s * stage_bytes;
    TA* sv = reinterpret_cast<TA*>(st);
    const int* sc = reinterpret_cast<const int*>(st + val_bytes);
    const int* sp = reinterpret_cast<const int*>(st + val_bytes + col_bytes);
    const int r0 = trow[t], r1 = trow[t + 1];
    const int p0 = r0 / 4 * 4;
    const int n0 = sp[r0 - p0], n1 = sp[r1 - p0];
    const int va0 = n0 / VA * VA, c0 = n0 / 4 * 4;
    // products of the whole tile in place, consecutive entries per thread
    // group (conflict-free), eight x-gathers in flight per thread
    for (int q0 = n0 + ct; q0 < n1; q0 += 8 * NC) {
      TX xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * NC;
        xv[u] = x[q < n1 ? sc[q - c0] : 0];
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * NC;
        if (q < n1) sv[q - va0] = TA(TACC(sv[q - va0]) * TACC(xv[u]));
      }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(NC) : "memory");  // consumer warps only
    // each row summed in its stored order by one thread
    for (int r = r0 + ct; r < r1; r += NC) {
      const int a = sp[r - p0], e = sp[r + 1 - p0];
      TACC sum = TACC(0);
      for (int q = a; q < e; ++q) sum += TACC(sv[q - va0]);
      if (MODE == SPMV_SET) {
        y[r] = TY(sum);
      } else if (MODE == SPMV_RES) {
        y[r] = TY(TACC(b[r]) - sum);
      } else if (MODE == SPMV_ADD) {
        y[r] = TY(TACC(y[r]) + sum);
      } else {
        const TACC sc2 = TACC(kind[r] == 1 ? s1 : s0);
        y[r] = TY(sc2 * (TACC(b[r]) - sum));
      }
    }
    asm volatile("bar.sync 1, %0;" ::"r"(NC) : "memory");
    if (lane == 0) mbar_arrive(empty + s);
  }
}

size_t spmv_tma_smem(const DevCSR& A) { return 128 + 3 * (size_t)(A.tile_val_bytes + A.tile_col_bytes + A.tile_rp_bytes); }

template <typename TA, typename TX, typename TB, typename TY, typename TACC>
cudaError_t spmv_tma(const DevCSR& A, const TA* val, const TX* x, const TB* b, TY* y, int mode, double s0, double s1,
                     const uint8_t* kind, cudaStream_t st) {
  const int vbytes = sizeof(TA) == 8 ? A.tile_val_bytes : A.tile_val_bytes32;
  const size_t shm = 128 + 3 * (size_t)(vbytes + A.tile_col_bytes + A.tile_rp_bytes);
  const int grid = sizeof(TA) == 8 ? A.tma_grid64 : A.tma_grid32;
#define SD_LAUNCH(M)                                                                                          \
  k_spmv_tma<TA, TX, TB, TY, TACC, M><<<grid, 32 * (kSpNCW + 1), shm, st>>>(                                   \
      A.ntiles, A.trow, A.rowptr, A.col, val, x, b, y, s0, s1, kind, vbytes, A.tile_col_bytes, A.tile_rp_bytes, \
      A.err)
  switch (mode) {
    case SPMV_SET: SD_LAUNCH(SPMV_SET); break;
    case SPMV_RES: SD_LAUNCH(SPMV_RES); break;
    case SPMV_ADD: SD_LAUNCH(SPMV_ADD); break;
    default: SD_LAUNCH(SPMV_SCALED_RES);
  }
#undef SD_LAUNCH
  return cudaGetLastError();
}

template <typename TA, typename TX, typename TB, typename TY, typename TACC>
static cudaError_t prep_one() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const void* ks[] = {(const void*)k_spmv_tma<TA, TX, TB, TY, TACC, SPMV_SET>,
                      (const void*)k_spmv_tma<TA, TX, TB, TY, TACC, SPMV_RES>,
                      (const void*)k_spmv_tma<TA, TX, TB, TY, TACC, SPMV_ADD>,
                      (const void*)k_spmv_tma<TA, TX, TB, TY, TACC, SPMV_SCALED_RES>};
  for (const void* k : ks)
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  return e;
}

#define SD_SPMV_TMA(TA, TX, TB, TY, TACC)                                                                    \
  template cudaError_t spmv_tma<TA, TX, TB, TY, TACC>(const DevCSR&, const TA*, const TX*, const TB*, TY*, int, \
                                                      double, double, const uint8_t*, cudaStream_t);
SD_SPMV_TMA(float, float, float, float, float)
SD_SPMV_TMA(double, double, double, double, double)
SD_SPMV_TMA(double, float, double, float, double)
SD_SPMV_TMA(double, float, float, float, double)
SD_SPMV_TMA(double, double, double, float, double)
SD_SPMV_TMA(float, float, double, float, float)
SD_SPMV_TMA(double, float, double, double, double)
#undef SD_SPMV_TMA

cudaError_t spmv_prepare_kernels() {
  cudaError_t e = prep_one<float, float, float, float, float>();
  if (e == cudaSuccess) e = prep_one<double, double, double, double, double>();
  if (e == cudaSuccess) e = prep_one<double, float, double, float, double>();
  if (e == cudaSuccess) e = prep_one<double, float, float, float, double>();
  if (e == cudaSuccess) e = prep_one<double, double, double, float, double>();
  if (e == cudaSuccess) e = prep_one<float, float, double, float, float>();
  if (e == cudaSuccess) e = prep_one<double, float, double, double, double>();
  return e;
}

int spmv_tma_blocks_per_sm(const DevCSR& A, bool fp64) {
  const int vbytes = fp64 ? A.tile_val_bytes : A.tile_val_bytes32;
  const size_t shm = 128 + 3 * (size_t)(vbytes + A.tile_col_bytes + A.tile_rp_bytes);
  int nb = 0;
  cudaError_t e = fp64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &nb, k_spmv_tma<double, double, double, double, double, SPMV_RES>, 32 * (kSpNCW + 1), shm)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             &nb, k_spmv_tma<float, float, float, float, float, SPMV_RES>, 32 * (kSpNCW + 1), shm);
  return e == cudaSuccess ? nb : 0;
}

}  // namespace sd
