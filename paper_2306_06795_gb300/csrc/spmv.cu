// Vector-CSR sparse matrix-vector products for every level operator, the
// transfers and the FP64 defect-correction residual (steps a1-a3).
// TPR threads cooperate on a row; the group size is chosen from the mean
// row length so that a warp streams contiguous values and columns.
#include <algorithm>

#include "common.cuh"

namespace sd {

template <typename TA, typename TX, typename TB, typename TY, typename TACC, int TPR, int MODE>
__global__ void __launch_bounds__(256) k_spmv(int nrows, const int* __restrict__ rowptr,
                                              const int* __restrict__ col, const TA* __restrict__ val,
                                              const TX* __restrict__ x, const TB* __restrict__ b,
                                              TY* __restrict__ y, double s0, double s1,
                                              const uint8_t* __restrict__ kind) {
  pdl_enter();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = tid / TPR;
  const int lane = (int)(tid % TPR);
  const bool valid = row < nrows;
  TACC sum = TACC(0);
  if (valid) {
    const int beg = __ldg(rowptr + row), end = __ldg(rowptr + row + 1);
    for (int k = beg + lane; k < end; k += TPR) sum += TACC(__ldg(val + k)) * TACC(x[__ldg(col + k)]);
  }
#pragma unroll
  for (int off = TPR / 2; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off, TPR);
  if (valid && lane == 0) {
    if (MODE == SPMV_SET) {
      y[row] = TY(sum);
    } else if (MODE == SPMV_RES) {
      y[row] = TY(TACC(b[row]) - sum);
    } else if (MODE == SPMV_ADD) {
      y[row] = TY(TACC(y[row]) + sum);
    } else {
      const TACC s = TACC(kind[row] == 1 ? s1 : s0);
      y[row] = TY(s * (TACC(b[row]) - sum));
    }
  }
}

template <typename TA, typename TX, typename TB, typename TY, typename TACC, int TPR>
static cudaError_t launch_mode(const DevCSR& A, const TA* val, const TX* x, const TB* b, TY* y, int mode,
                               double s0, double s1, const uint8_t* kind, cudaStream_t st) {
  if (A.nrows == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t total = (int64_t)A.nrows * TPR;
  const unsigned blocks = (unsigned)((total + threads - 1) / threads);
  switch (mode) {
    case SPMV_SET:
      SD_LAUNCH((k_spmv<TA, TX, TB, TY, TACC, TPR, SPMV_SET>), blocks, threads, 0, st, A.nrows, A.rowptr, A.col, val, x, b, y, s0, s1, kind);
      break;
    case SPMV_RES:
      SD_LAUNCH((k_spmv<TA, TX, TB, TY, TACC, TPR, SPMV_RES>), blocks, threads, 0, st, A.nrows, A.rowptr, A.col, val, x, b, y, s0, s1, kind);
      break;
    case SPMV_ADD:
      SD_LAUNCH((k_spmv<TA, TX, TB, TY, TACC, TPR, SPMV_ADD>), blocks, threads, 0, st, A.nrows, A.rowptr, A.col, val, x, b, y, s0, s1, kind);
      break;
    default:
      SD_LAUNCH((k_spmv<TA, TX, TB, TY, TACC, TPR, SPMV_SCALED_RES>), blocks, threads, 0, st, A.nrows, A.rowptr, A.col, val, x, b, y, s0, s1, kind);
  }
  return cudaGetLastError();
}

// Sliced-ELLPACK product: a warp owns a chunk of 32 consecutive rows, one
// row per lane, so at step k the warp reads 32 consecutive values and
// columns (one coalesced line each, streamed past L2) and gathers x through
// the read-only path.  Padding entries carry column -1 and are skipped, so
// no row lengths are read.  U steps (8 for FP32 values, 4 for FP64) have
// their values and columns in flight together, then their x gathers; this
// beat a software-pipelined variant and two rows per lane on the C2 level
// operators.  Each row sums its entries in CSR order.
constexpr int kSellWarps = 8;

template <typename TA, typename TX, typename TB, typename TY, typename TACC, int MODE>
__global__ void __launch_bounds__(32 * kSellWarps) k_spmv_sell(int nrows, int nchunks,
    const int64_t* __restrict__ soff, const int* __restrict__ scol, const TA* __restrict__ sval,
    const TX* __restrict__ x, const TB* __restrict__ b, TY* __restrict__ y, double s0, double s1,
    const uint8_t* __restrict__ kind) {
  pdl_enter();
  const int c = blockIdx.x * kSellWarps + (threadIdx.x >> 5);
  if (c >= nchunks) return;
  const int lane = threadIdx.x & 31;
  const int row = c * 32 + lane;
  const int64_t o0 = soff[c];
  const int w = (int)((soff[c + 1] - o0) >> 5);  // uniform over the warp
  const TA* vp = sval + o0 + lane;
  const int* cp = scol + o0 + lane;
  constexpr int U = sizeof(TA) == 4 ? 8 : 4;
  TACC sum = TACC(0);
  for (int k = 0; k < w; k += U) {
    TA v[U];
    int cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int kk = k + u;
      v[u] = kk < w ? __ldcs(vp + (int64_t)kk * 32) : TA(0);
      cc[u] = kk < w ? __ldcs(cp + (int64_t)kk * 32) : -1;
    }
    TX xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = cc[u] >= 0 ? __ldg(x + cc[u]) : TX(0);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (cc[u] >= 0) sum += TACC(v[u]) * TACC(xv[u]);
  }
  if (row >= nrows) return;
  if (MODE == SPMV_SET) {
    y[row] = TY(sum);
  } else if (MODE == SPMV_RES) {
    y[row] = TY(TACC(b[row]) - sum);
  } else if (MODE == SPMV_ADD) {
    y[row] = TY(TACC(y[row]) + sum);
  } else {
    const TACC sc = TACC(kind[row] == 1 ? s1 : s0);
    y[row] = TY(sc * (TACC(b[row]) - sum));
  }
}

// Row-block ("stream") product: a block of 256 threads owns a tile of
// consecutive rows holding at most kStreamNnz stored entries (cut at setup;
// the tile descriptor {first row, first entry, end row, end entry} is one
// 16-byte load).  Every thread loads eight of the tile's values and columns
// at once (coalesced, streamed past L2) together with the tile's row
// pointers, then gathers the eight x entries at once and stages values and
// x entries in shared memory; after one barrier thread i sums row i of the
// tile in CSR order, one FMA per entry (one DFMA in FP64, whose rate is low
// on GB300).  Three memory round trips per tile and 16-32 KB of loads in
// flight per block, whatever the row lengths.
constexpr int kStreamThreads = 256;

template <typename TA, typename TX, typename TB, typename TY, typename TACC, int MODE>
__global__ void __launch_bounds__(kStreamThreads) k_spmv_stream(const int4* __restrict__ tdesc,
    const int* __restrict__ rowptr, const int* __restrict__ col, const TA* __restrict__ val,
    const TX* __restrict__ x, const TB* __restrict__ b, TY* __restrict__ y, double s0, double s1,
    const uint8_t* __restrict__ kind) {
  pdl_enter();
  constexpr int PER = kStreamNnz / kStreamThreads;
  __shared__ TA sv[kStreamNnz];
  __shared__ TX sx[kStreamNnz];
  __shared__ int srp[kStreamRows + 1];
  const int4 d = tdesc[blockIdx.x];
  const int r0 = d.x, e0 = d.y, nr = d.z - d.x, ne = d.w - d.y;
  const int tid = threadIdx.x;
  TA v[PER];
  int cc[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int q = u * kStreamThreads + tid;
    v[u] = q < ne ? __ldcs(val + e0 + q) : TA(0);
    cc[u] = q < ne ? __ldcs(col + e0 + q) : -1;
  }
  for (int i = tid; i <= nr; i += kStreamThreads) srp[i] = rowptr[r0 + i] - e0;
  TB bv = TB(0);
  uint8_t kv = 0;
  if (tid < nr) {
    if (MODE == SPMV_RES || MODE == SPMV_SCALED_RES) bv = b[r0 + tid];
    if (MODE == SPMV_SCALED_RES) kv = kind[r0 + tid];
  }
  TX xv[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) xv[u] = cc[u] >= 0 ? __ldg(x + cc[u]) : TX(0);
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    sv[u * kStreamThreads + tid] = v[u];
    sx[u * kStreamThreads + tid] = xv[u];
  }
  __syncthreads();
  if (tid >= nr) return;
  TACC sum = TACC(0);
  const int q1 = srp[tid + 1];
  for (int q = srp[tid]; q < q1; ++q) sum = fma(TACC(sv[q]), TACC(sx[q]), sum);
  const int row = r0 + tid;
  if (MODE == SPMV_SET) {
    y[row] = TY(sum);
  } else if (MODE == SPMV_RES) {
    y[row] = TY(TACC(bv) - sum);
  } else if (MODE == SPMV_ADD) {
    y[row] = TY(TACC(y[row]) + sum);
  } else {
    const TACC sc = TACC(kv == 1 ? s1 : s0);
    y[row] = TY(sc * (TACC(bv) - sum));
  }
}

template <typename TA, typename TX, typename TB, typename TY, typename TACC>
static cudaError_t spmv_stream(const DevCSR& A, const TA* val, const TX* x, const TB* b, TY* y, int mode, double s0,
                               double s1, const uint8_t* kind, cudaStream_t st) {
  const unsigned blocks = (unsigned)A.stiles;
  switch (mode) {
    case SPMV_SET:
      SD_LAUNCH((k_spmv_stream<TA, TX, TB, TY, TACC, SPMV_SET>), blocks, kStreamThreads, 0, st, A.tdesc, A.rowptr, A.col, val, x, b, y, s0, s1, kind);
      break;
    case SPMV_RES:
      SD_LAUNCH((k_spmv_stream<TA, TX, TB, TY, TACC, SPMV_RES>), blocks, kStreamThreads, 0, st, A.tdesc, A.rowptr, A.col, val, x, b, y, s0, s1, kind);
      break;
    case SPMV_ADD:
      SD_LAUNCH((k_spmv_stream<TA, TX, TB, TY, TACC, SPMV_ADD>), blocks, kStreamThreads, 0, st, A.tdesc, A.rowptr, A.col, val, x, b, y, s0, s1, kind);
      break;
    default:
      SD_LAUNCH((k_spmv_stream<TA, TX, TB, TY, TACC, SPMV_SCALED_RES>), blocks, kStreamThreads, 0, st, A.tdesc, A.rowptr, A.col, val, x, b, y, s0, s1, kind);
  }
  return cudaGetLastError();
}

template <typename TA> const TA* sell_values(const DevCSR& A);
template <> const float* sell_values<float>(const DevCSR& A) { return A.sv32; }
template <> const double* sell_values<double>(const DevCSR& A) { return A.sv64; }

template <typename TA, typename TX, typename TB, typename TY, typename TACC>
static cudaError_t spmv_sell(const DevCSR& A, const TA* sval, const TX* x, const TB* b, TY* y, int mode, double s0,
                             double s1, const uint8_t* kind, cudaStream_t st) {
  const unsigned blocks = (unsigned)((A.schunks + kSellWarps - 1) / kSellWarps);
  const int threads = 32 * kSellWarps;
  switch (mode) {
    case SPMV_SET:
      SD_LAUNCH((k_spmv_sell<TA, TX, TB, TY, TACC, SPMV_SET>), blocks, threads, 0, st, A.nrows, A.schunks, A.soff, A.scol, sval, x, b, y, s0, s1, kind);
      break;
    case SPMV_RES:
      SD_LAUNCH((k_spmv_sell<TA, TX, TB, TY, TACC, SPMV_RES>), blocks, threads, 0, st, A.nrows, A.schunks, A.soff, A.scol, sval, x, b, y, s0, s1, kind);
      break;
    case SPMV_ADD:
      SD_LAUNCH((k_spmv_sell<TA, TX, TB, TY, TACC, SPMV_ADD>), blocks, threads, 0, st, A.nrows, A.schunks, A.soff, A.scol, sval, x, b, y, s0, s1, kind);
      break;
    default:
      SD_LAUNCH((k_spmv_sell<TA, TX, TB, TY, TACC, SPMV_SCALED_RES>), blocks, threads, 0, st, A.nrows, A.schunks, A.soff, A.scol, sval, x, b, y, s0, s1, kind);
  }
  return cudaGetLastError();
}

template <typename TA, typename TX, typename TB, typename TY, typename TACC>
cudaError_t spmv(const DevCSR& A, const TA* val, const TX* x, const TB* b, TY* y, int mode, double s0,
                 double s1, const uint8_t* kind, cudaStream_t st) {
  if (A.stiles > 0) return spmv_stream<TA, TX, TB, TY, TACC>(A, val, x, b, y, mode, s0, s1, kind, st);
  // the sliced copy holds the same values as A.v32 / A.v64
  if (A.schunks > 0 && sell_values<TA>(A) && (const void*)val == (const void*)(sizeof(TA) == 4 ? (const void*)A.v32 : (const void*)A.v64))
    return spmv_sell<TA, TX, TB, TY, TACC>(A, sell_values<TA>(A), x, b, y, mode, s0, s1, kind, st);
  switch (A.tpr) {
    case 2: return launch_mode<TA, TX, TB, TY, TACC, 2>(A, val, x, b, y, mode, s0, s1, kind, st);
    case 4: return launch_mode<TA, TX, TB, TY, TACC, 4>(A, val, x, b, y, mode, s0, s1, kind, st);
    case 8: return launch_mode<TA, TX, TB, TY, TACC, 8>(A, val, x, b, y, mode, s0, s1, kind, st);
    case 16: return launch_mode<TA, TX, TB, TY, TACC, 16>(A, val, x, b, y, mode, s0, s1, kind, st);
    default: return launch_mode<TA, TX, TB, TY, TACC, 32>(A, val, x, b, y, mode, s0, s1, kind, st);
  }
}

// y = R b - (R K) x, both sums of a coarse row by the same TPR lanes (each
// in CSR order per lane, then a fixed shuffle tree).
template <typename T, int TPR>
__global__ void __launch_bounds__(256) k_restrict_res(int nrows, const int* __restrict__ rp, const int* __restrict__ rc,
                                                      const T* __restrict__ rv, const T* __restrict__ b,
                                                      const int* __restrict__ kp, const int* __restrict__ kc,
                                                      const T* __restrict__ kv, const T* __restrict__ x,
                                                      T* __restrict__ y) {
  pdl_enter();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = tid / TPR;
  const int lane = (int)(tid % TPR);
  const bool valid = row < nrows;
  T s1 = T(0), s2 = T(0);
  if (valid) {
    for (int k = rp[row] + lane; k < rp[row + 1]; k += TPR) s1 += rv[k] * b[rc[k]];
    for (int k = kp[row] + lane; k < kp[row + 1]; k += TPR) s2 += kv[k] * x[kc[k]];
  }
#pragma unroll
  for (int off = TPR / 2; off > 0; off >>= 1) {
    s1 += __shfl_down_sync(0xffffffffu, s1, off, TPR);
    s2 += __shfl_down_sync(0xffffffffu, s2, off, TPR);
  }
  if (valid && lane == 0) y[row] = s1 - s2;
}

template <typename T>
cudaError_t restrict_res(const DevCSR& R, const T* rval, const T* b, const DevCSR& RK, const T* rkval, const T* x,
                         T* y, cudaStream_t st) {
  if (R.nrows == 0) return cudaSuccess;
  if (RK.nrows != R.nrows) return cudaErrorInvalidValue;
  const int tpr = std::max(R.tpr, RK.tpr);
  const int64_t total = (int64_t)R.nrows * tpr;
  const unsigned blocks = (unsigned)((total + 255) / 256);
#define SD_RR(TP) SD_LAUNCH((k_restrict_res<T, TP>), blocks, 256, 0, st, R.nrows, R.rowptr, R.col, rval, b, RK.rowptr, RK.col, rkval, x, y)
  switch (tpr) {
    case 2: SD_RR(2); break;
    case 4: SD_RR(4); break;
    case 8: SD_RR(8); break;
    case 16: SD_RR(16); break;
    default: SD_RR(32); break;
  }
#undef SD_RR
  return cudaGetLastError();
}
template cudaError_t restrict_res<float>(const DevCSR&, const float*, const float*, const DevCSR&, const float*,
                                         const float*, float*, cudaStream_t);
template cudaError_t restrict_res<double>(const DevCSR&, const double*, const double*, const DevCSR&, const double*,
                                          const double*, double*, cudaStream_t);

#define SD_SPMV(TA, TX, TB, TY, TACC)                                                                  \
  template cudaError_t spmv<TA, TX, TB, TY, TACC>(const DevCSR&, const TA*, const TX*, const TB*, TY*, \
                                                  int, double, double, const uint8_t*, cudaStream_t);
SD_SPMV(float, float, float, float, float)
SD_SPMV(double, double, double, double, double)
SD_SPMV(double, float, double, float, double)   // FP64 DC residual of an FP32 cycle
SD_SPMV(double, float, float, float, double)
SD_SPMV(double, double, double, float, double)
SD_SPMV(float, float, double, float, float)
SD_SPMV(double, float, double, double, double)   // FP64 DC residual into an FP64 buffer
#undef SD_SPMV

}  // namespace sd
