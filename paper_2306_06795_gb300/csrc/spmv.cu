// Vector-CSR sparse matrix-vector products for every level operator, the
// transfers and the FP64 defect-correction residual (steps a1-a3).
// TPR threads cooperate on a row; the group size is chosen from the mean
// row length so that a warp streams contiguous values and columns.
#include "common.cuh"

namespace sd {

template <typename TA, typename TX, typename TB, typename TY, typename TACC, int TPR, int MODE>
__global__ void __launch_bounds__(256) k_spmv(int nrows, const int* __restrict__ rowptr,
                                              const int* __restrict__ col, const TA* __restrict__ val,
                                              const TX* __restrict__ x, const TB* __restrict__ b,
                                              TY* __restrict__ y, double s0, double s1,
                                              const uint8_t* __restrict__ kind) {
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
      k_spmv<TA, TX, TB, TY, TACC, TPR, SPMV_SET><<<blocks, threads, 0, st>>>(A.nrows, A.rowptr, A.col, val, x, b, y, s0, s1, kind);
      break;
    case SPMV_RES:
      k_spmv<TA, TX, TB, TY, TACC, TPR, SPMV_RES><<<blocks, threads, 0, st>>>(A.nrows, A.rowptr, A.col, val, x, b, y, s0, s1, kind);
      break;
    case SPMV_ADD:
      k_spmv<TA, TX, TB, TY, TACC, TPR, SPMV_ADD><<<blocks, threads, 0, st>>>(A.nrows, A.rowptr, A.col, val, x, b, y, s0, s1, kind);
      break;
    default:
      k_spmv<TA, TX, TB, TY, TACC, TPR, SPMV_SCALED_RES><<<blocks, threads, 0, st>>>(A.nrows, A.rowptr, A.col, val, x, b, y, s0, s1, kind);
  }
  return cudaGetLastError();
}

template <typename TA, typename TX, typename TB, typename TY, typename TACC>
cudaError_t spmv(const DevCSR& A, const TA* val, const TX* x, const TB* b, TY* y, int mode, double s0,
                 double s1, const uint8_t* kind, cudaStream_t st) {
  if (A.ntiles > 0) return spmv_tma<TA, TX, TB, TY, TACC>(A, val, x, b, y, mode, s0, s1, kind, st);
  switch (A.tpr) {
    case 2: return launch_mode<TA, TX, TB, TY, TACC, 2>(A, val, x, b, y, mode, s0, s1, kind, st);
    case 4: return launch_mode<TA, TX, TB, TY, TACC, 4>(A, val, x, b, y, mode, s0, s1, kind, st);
    case 8: return launch_mode<TA, TX, TB, TY, TACC, 8>(A, val, x, b, y, mode, s0, s1, kind, st);
    case 16: return launch_mode<TA, TX, TB, TY, TACC, 16>(A, val, x, b, y, mode, s0, s1, kind, st);
    default: return launch_mode<TA, TX, TB, TY, TACC, 32>(A, val, x, b, y, mode, s0, s1, kind, st);
  }
}

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
