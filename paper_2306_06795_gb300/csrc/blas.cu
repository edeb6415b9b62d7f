// Elementwise kernels, the coarsest exact solve (step a9) and the
// segmented deterministic reductions of the FP64 FGMRES (step a11).
// Every reduction has a fixed decomposition (chunks of rows, then a fixed
// tree inside a block, then chunks summed in ascending order), so results
// are bitwise reproducible run to run.
#include "common.cuh"

namespace sd {

template <typename TI, typename TO>
__global__ void k_cast(int64_t n, const TI* __restrict__ in, TO* __restrict__ out) {
  pdl_enter();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = TO(in[j]);
}
template <typename TI, typename TO>
cudaError_t cast_copy(int64_t n, const TI* in, TO* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  SD_LAUNCH((k_cast<TI, TO>), (unsigned)((n + 255) / 256), 256, 0, st, n, in, out);
  return cudaGetLastError();
}
template cudaError_t cast_copy<double, float>(int64_t, const double*, float*, cudaStream_t);
template cudaError_t cast_copy<float, double>(int64_t, const float*, double*, cudaStream_t);
template cudaError_t cast_copy<double, double>(int64_t, const double*, double*, cudaStream_t);
template cudaError_t cast_copy<float, float>(int64_t, const float*, float*, cudaStream_t);

template <typename T, typename TI>
__global__ void k_axpy(int64_t n, T a, const TI* __restrict__ x, T* __restrict__ y) {
  pdl_enter();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) y[j] += a * T(x[j]);
}
template <typename T, typename TI>
cudaError_t axpy_into(int64_t n, double a, const TI* x, T* y, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  SD_LAUNCH((k_axpy<T, TI>), (unsigned)((n + 255) / 256), 256, 0, st, n, T(a), x, y);
  return cudaGetLastError();
}
template cudaError_t axpy_into<float, float>(int64_t, double, const float*, float*, cudaStream_t);
template cudaError_t axpy_into<double, double>(int64_t, double, const double*, double*, cudaStream_t);
template cudaError_t axpy_into<double, float>(int64_t, double, const float*, double*, cudaStream_t);

template <typename T>
__global__ void k_zero(int64_t n, T* __restrict__ y) {
  pdl_enter();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) y[j] = T(0);
}
template <typename T>
cudaError_t fill_zero(int64_t n, T* y, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  SD_LAUNCH(k_zero<T>, (unsigned)((n + 255) / 256), 256, 0, st, n, y);
  return cudaGetLastError();
}
template cudaError_t fill_zero<float>(int64_t, float*, cudaStream_t);
template cudaError_t fill_zero<double>(int64_t, double*, cudaStream_t);

// z = d .* u (the Jacobi step inside a Krylov-wrapped relaxation)
template <typename T>
__global__ void k_diag_scale(int64_t n, const T* __restrict__ d, const T* __restrict__ u, T* __restrict__ z) {
  pdl_enter();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) z[j] = d[j] * u[j];
}
template <typename T>
cudaError_t diag_scale(int64_t n, const T* d, const T* u, T* z, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  SD_LAUNCH(k_diag_scale<T>, (unsigned)((n + 255) / 256), 256, 0, st, n, d, u, z);
  return cudaGetLastError();
}
template cudaError_t diag_scale<float>(int64_t, const float*, const float*, float*, cudaStream_t);
template cudaError_t diag_scale<double>(int64_t, const double*, const double*, double*, cudaStream_t);

// BTP output in FP64: velocity rows take du (Dirichlet rows r), pressure
// rows sp * dp.
template <typename T>
__global__ void k_btp_out(int64_t nu, int64_t np, const T* __restrict__ du, const T* __restrict__ dp, double sp,
                          const uint8_t* __restrict__ dir, const double* __restrict__ r64, double* __restrict__ z) {
  pdl_enter();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nu) z[j] = dir[j] ? r64[j] : (double)du[j];
  else if (j < nu + np) z[j] = sp * (double)dp[j - nu];
}
template <typename T>
cudaError_t btp_out(int64_t nu, int64_t np, const T* du, const T* dp, double sp, const uint8_t* dir,
                    const double* r64, double* z, cudaStream_t st) {
  if (nu + np == 0) return cudaSuccess;
  SD_LAUNCH(k_btp_out<T>, (unsigned)((nu + np + 255) / 256), 256, 0, st, nu, np, du, dp, sp, dir, r64, z);
  return cudaGetLastError();
}
template cudaError_t btp_out<float>(int64_t, int64_t, const float*, const float*, double, const uint8_t*,
                                    const double*, double*, cudaStream_t);
template cudaError_t btp_out<double>(int64_t, int64_t, const double*, const double*, double, const uint8_t*,
                                     const double*, double*, cudaStream_t);

template <typename T>
__global__ void k_finalize(int64_t n, const T* __restrict__ x, const uint8_t* __restrict__ dir,
                           const double* __restrict__ r64, double* __restrict__ out) {
  pdl_enter();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = dir[j] ? r64[j] : double(x[j]);
}
template <typename T>
cudaError_t finalize_out(int64_t n, const T* x, const uint8_t* dir, const double* r64, double* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  SD_LAUNCH(k_finalize<T>, (unsigned)((n + 255) / 256), 256, 0, st, n, x, dir, r64, out);
  return cudaGetLastError();
}
template cudaError_t finalize_out<float>(int64_t, const float*, const uint8_t*, const double*, double*, cudaStream_t);
template cudaError_t finalize_out<double>(int64_t, const double*, const uint8_t*, const double*, double*, cudaStream_t);

__global__ void k_flush(int4* buf, int64_t n, int v) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    buf[j] = make_int4(v, v, v, v);
}
cudaError_t l2_flush(void* buf, size_t bytes, cudaStream_t st) {
  k_flush<<<152 * 8, 256, 0, st>>>(reinterpret_cast<int4*>(buf), (int64_t)(bytes / 16), 1);
  return cudaGetLastError();
}

// ------------------------------------------------------------ Chebyshev
template <typename T>
__global__ void k_cheb_init(int64_t n, const T* __restrict__ b, const T* __restrict__ dinv,
                            const uint8_t* __restrict__ mask, uint8_t want, T s, T inv_theta, T* __restrict__ r,
                            T* __restrict__ d, T* __restrict__ x) {
  pdl_enter();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  T v = (!mask || mask[j] == want) ? s * b[j] : T(0);
  if (dinv) v *= dinv[j];
  r[j] = v;
  d[j] = v * inv_theta;
  x[j] = T(0);
}
template <typename T>
cudaError_t cheb_init(int64_t n, const T* b, const T* dinv, const uint8_t* mask, uint8_t want, double s, double theta,
                      T* r, T* d, T* x, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  SD_LAUNCH(k_cheb_init<T>, (unsigned)((n + 255) / 256), 256, 0, st, n, b, dinv, mask, want, T(s), T(1.0 / theta), r, d, x);
  return cudaGetLastError();
}
template cudaError_t cheb_init<float>(int64_t, const float*, const float*, const uint8_t*, uint8_t, double, double,
                                      float*, float*, float*, cudaStream_t);
template cudaError_t cheb_init<double>(int64_t, const double*, const double*, const uint8_t*, uint8_t, double, double,
                                       double*, double*, double*, cudaStream_t);

// Both Chebyshev steps on the sliced-ELLPACK copy of M (a warp owns 32
// consecutive rows, one per lane, values and columns of step k of the 32
// rows contiguous; padding has column -1): STEP = 0 the plain step (w = d_in
// or B^T d, dinv optional), STEP = 1 / 2 the first step from b, x set / x
// accumulated.  Each row sums its entries in CSR order.
template <typename T, int STEP>
__global__ void __launch_bounds__(256) k_cheb_sell(int nrows, int nchunks, const int64_t* __restrict__ soff,
                                                   const int* __restrict__ scol, const T* __restrict__ sval,
                                                   const T* __restrict__ w, const T* __restrict__ dinv,
                                                   T* __restrict__ x, T* __restrict__ r, const T* __restrict__ din,
                                                   T* __restrict__ dout, T s, T c, T alpha, T beta) {
  pdl_enter();
  const int ch = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (ch >= nchunks) return;
  const int lane = threadIdx.x & 31;
  const int row = ch * 32 + lane;
  const int64_t o0 = soff[ch];
  const int wd = (int)((soff[ch + 1] - o0) >> 5);
  const T* vp = sval + o0 + lane;
  const int* cp = scol + o0 + lane;
  constexpr int U = sizeof(T) == 4 ? 8 : 4;
  T sum = T(0);
  for (int k = 0; k < wd; k += U) {
    T v[U];
    int cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int kk = k + u;
      v[u] = kk < wd ? __ldcs(vp + (int64_t)kk * 32) : T(0);
      cc[u] = kk < wd ? __ldcs(cp + (int64_t)kk * 32) : -1;
    }
    T xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = cc[u] >= 0 ? w[cc[u]] : T(0);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (cc[u] >= 0) sum += v[u] * xv[u];
  }
  if (row >= nrows) return;
  if (STEP == 0) {
    const T dv = din[row];
    x[row] += dv;
    const T rv = r[row] - (dinv ? dinv[row] * sum : sum);
    r[row] = rv;
    dout[row] = alpha * dv + beta * rv;
  } else {
    const T bv = w[row];
    const T d0 = c * bv;
    x[row] = STEP == 2 ? x[row] + d0 : d0;
    const T rv = s * bv - c * sum;
    r[row] = rv;
    dout[row] = alpha * d0 + beta * rv;
  }
}

template <typename T> static const T* sell_vals(const DevCSR& M);
template <> const float* sell_vals<float>(const DevCSR& M) { return M.sv32; }
template <> const double* sell_vals<double>(const DevCSR& M) { return M.sv64; }
// the sliced copy when M has one and val is M's own value array
template <typename T>
static bool use_sell(const DevCSR& M, const T* val) {
  return M.schunks > 0 && sell_vals<T>(M) && (const void*)val == (sizeof(T) == 4 ? (const void*)M.v32 : (const void*)M.v64);
}

template <typename T, int TPR>
__global__ void __launch_bounds__(256) k_cheb_step(int nrows, const int* __restrict__ rowptr,
                                                   const int* __restrict__ col, const T* __restrict__ val,
                                                   const T* __restrict__ w, const T* __restrict__ dinv,
                                                   T* __restrict__ x, T* __restrict__ r, const T* __restrict__ din,
                                                   T* __restrict__ dout, T alpha, T beta) {
  pdl_enter();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = tid / TPR;
  const int lane = (int)(tid % TPR);
  const bool valid = row < nrows;
  T sum = T(0);
  if (valid)
    for (int k = rowptr[row] + lane; k < rowptr[row + 1]; k += TPR) sum += val[k] * w[col[k]];
#pragma unroll
  for (int off = TPR / 2; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off, TPR);
  if (valid && lane == 0) {
    const T dv = din[row];
    x[row] += dv;
    const T rv = r[row] - (dinv ? dinv[row] * sum : sum);
    r[row] = rv;
    dout[row] = alpha * dv + beta * rv;
  }
}
template <typename T>
cudaError_t cheb_step(const DevCSR& M, const T* val, const T* w, const T* dinv, T* x, T* r, const T* d_in, T* d_out,
                      double alpha, double beta, cudaStream_t st) {
  if (M.nrows == 0) return cudaSuccess;
  if (use_sell<T>(M, val)) {
    const unsigned blocks = (unsigned)((M.schunks + 7) / 8);
    SD_LAUNCH((k_cheb_sell<T, 0>), blocks, 256, 0, st, M.nrows, M.schunks, M.soff, M.scol, sell_vals<T>(M), w, dinv,
              x, r, d_in, d_out, T(0), T(0), T(alpha), T(beta));
    return cudaGetLastError();
  }
  const int64_t total = (int64_t)M.nrows * 8;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  SD_LAUNCH((k_cheb_step<T, 8>), blocks, 256, 0, st, M.nrows, M.rowptr, M.col, val, w, dinv, x, r, d_in, d_out, T(alpha), T(beta));
  return cudaGetLastError();
}
template <typename T, int TPR, bool ACC>
__global__ void __launch_bounds__(256) k_cheb_first(int nrows, const int* __restrict__ rowptr,
                                                    const int* __restrict__ col, const T* __restrict__ val,
                                                    const T* __restrict__ b, T s, T c, T* __restrict__ x,
                                                    T* __restrict__ r, T* __restrict__ dout, T alpha, T beta) {
  pdl_enter();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = tid / TPR;
  const int lane = (int)(tid % TPR);
  const bool valid = row < nrows;
  T sum = T(0);
  if (valid)
    for (int k = rowptr[row] + lane; k < rowptr[row + 1]; k += TPR) sum += val[k] * b[col[k]];
#pragma unroll
  for (int off = TPR / 2; off > 0; off >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, off, TPR);
  if (valid && lane == 0) {
    const T bv = b[row];
    const T d0 = c * bv;  // d0 = (s / theta) b;  M d0 = c M b
    x[row] = ACC ? x[row] + d0 : d0;
    const T rv = s * bv - c * sum;
    r[row] = rv;
    dout[row] = alpha * d0 + beta * rv;
  }
}
template <typename T>
cudaError_t cheb_first(const DevCSR& M, const T* val, const T* b, double s, double theta, T* x, T* r, T* d_out,
                       double alpha, double beta, bool accumulate, cudaStream_t st) {
  if (M.nrows == 0) return cudaSuccess;
  if (use_sell<T>(M, val)) {
    const unsigned blocks = (unsigned)((M.schunks + 7) / 8);
    if (accumulate)
      SD_LAUNCH((k_cheb_sell<T, 2>), blocks, 256, 0, st, M.nrows, M.schunks, M.soff, M.scol, sell_vals<T>(M), b,
                (const T*)nullptr, x, r, (const T*)nullptr, d_out, T(s), T(s / theta), T(alpha), T(beta));
    else
      SD_LAUNCH((k_cheb_sell<T, 1>), blocks, 256, 0, st, M.nrows, M.schunks, M.soff, M.scol, sell_vals<T>(M), b,
                (const T*)nullptr, x, r, (const T*)nullptr, d_out, T(s), T(s / theta), T(alpha), T(beta));
    return cudaGetLastError();
  }
  const int64_t total = (int64_t)M.nrows * 8;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  if (accumulate)
    SD_LAUNCH((k_cheb_first<T, 8, true>), blocks, 256, 0, st, M.nrows, M.rowptr, M.col, val, b, T(s), T(s / theta), x,
              r, d_out, T(alpha), T(beta));
  else
    SD_LAUNCH((k_cheb_first<T, 8, false>), blocks, 256, 0, st, M.nrows, M.rowptr, M.col, val, b, T(s), T(s / theta), x,
              r, d_out, T(alpha), T(beta));
  return cudaGetLastError();
}
template cudaError_t cheb_first<float>(const DevCSR&, const float*, const float*, double, double, float*, float*,
                                       float*, double, double, bool, cudaStream_t);
template cudaError_t cheb_first<double>(const DevCSR&, const double*, const double*, double, double, double*, double*,
                                        double*, double, double, bool, cudaStream_t);
template cudaError_t cheb_step<float>(const DevCSR&, const float*, const float*, const float*, float*, float*,
                                      const float*, float*, double, double, cudaStream_t);
template cudaError_t cheb_step<double>(const DevCSR&, const double*, const double*, const double*, double*, double*,
                                       const double*, double*, double, double, cudaStream_t);

template <typename TI, typename TO>
__global__ void k_scatter_rows(int64_t n, const TI* __restrict__ in, const int* __restrict__ rows, TO* __restrict__ out) {
  pdl_enter();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[rows[j]] = TO(in[j]);
}
template <typename TI, typename TO>
cudaError_t scatter_rows(int64_t n, const TI* in, const int* rows, TO* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  SD_LAUNCH((k_scatter_rows<TI, TO>), (unsigned)((n + 255) / 256), 256, 0, st, n, in, rows, out);
  return cudaGetLastError();
}
template cudaError_t scatter_rows<double, float>(int64_t, const double*, const int*, float*, cudaStream_t);
template cudaError_t scatter_rows<double, double>(int64_t, const double*, const int*, double*, cudaStream_t);

// ------------------------------------------------------------ coarse solve
// One warp per output row; grid.y runs over the coarse blocks (instances).
template <typename T>
__global__ void __launch_bounds__(128) k_coarse(const int* __restrict__ boff, const int* __restrict__ bn,
                                                const int64_t* __restrict__ koff, const double* __restrict__ Kinv,
                                                const T* __restrict__ b, T* __restrict__ y) {
  pdl_enter();
  const int kb = blockIdx.y;
  const int n = bn[kb];
  const int row = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const int off = boff[kb];
  const double* Krow = Kinv + koff[kb] + (int64_t)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += Krow[j] * double(b[off + j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[off + row] = T(s);
}
template <typename T>
cudaError_t coarse_solve(int nblocks, const int* boff, const int* bn, const int64_t* koff, const double* Kinv,
                         int max_n, const T* b, T* y, cudaStream_t st) {
  if (nblocks == 0) return cudaSuccess;
  dim3 grid((unsigned)((max_n + 3) / 4), (unsigned)nblocks);
  SD_LAUNCH((k_coarse<T>), grid, 128, 0, st, boff, bn, koff, Kinv, b, y);
  return cudaGetLastError();
}
template cudaError_t coarse_solve<float>(int, const int*, const int*, const int64_t*, const double*, int,
                                         const float*, float*, cudaStream_t);
template cudaError_t coarse_solve<double>(int, const int*, const int*, const int64_t*, const double*, int,
                                          const double*, double*, cudaStream_t);

// ------------------------------------------------------------ reductions
constexpr int kRedThreads = 256;
constexpr int kMaxAxpyCols = 1024;  // Krylov columns (restart length) one multiaxpy handles

// grid: (nchunks, ceil(ncols / NK)).  partial[c*ldp + k] = sum over the
// rows of chunk c of V_k[row] w[row] for NK columns k per block (NK = 1, 2,
// 4 or 8, the smallest power of two covering ncols, at most 8): two rows
// per thread per step with all column loads in flight, one DFMA per loaded
// element (columns past ncols are neither loaded nor multiplied: GB300's
// FP64 rate is the bound), then a transposed butterfly that halves the
// values a lane holds at each of the first log2(NK) exchanges and adds in
// full at the others (NK - 1 + 5 - log2(NK) additions per warp instead of
// 5 NK), and the warps' sums are added in warp order.  Fixed order:
// deterministic.
template <int NK>
__global__ void __launch_bounds__(kRedThreads, 4) k_multidot(const int64_t* __restrict__ cbeg,
    const int64_t* __restrict__ cend, int ncols, const double* __restrict__ V, int64_t ldv,
    const double* __restrict__ w, double* __restrict__ partial, int ldp) {
  pdl_enter();
  __shared__ double red[kRedThreads / 32][NK];
  const int c = blockIdx.x, k0 = blockIdx.y * NK;
  const int nk = min(NK, ncols - k0);
  double acc[NK];
#pragma unroll
  for (int u = 0; u < NK; ++u) acc[u] = 0.0;
  const double* v0 = V + (int64_t)k0 * ldv;
  const int64_t ce = cend[c];
  for (int64_t r = cbeg[c] + threadIdx.x; r < ce; r += 2 * kRedThreads) {
    const int64_t r2 = r + kRedThreads;
    const bool has2 = r2 < ce;
    const double w1 = w[r], w2 = has2 ? w[r2] : 0.0;
    double v1[NK], v2[NK];
#pragma unroll
    for (int u = 0; u < NK; ++u) {
      v1[u] = u < nk ? v0[(int64_t)u * ldv + r] : 0.0;
      v2[u] = u < nk && has2 ? v0[(int64_t)u * ldv + r2] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < NK; ++u)
      if (u < nk) acc[u] = fma(v2[u], w2, fma(v1[u], w1, acc[u]));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // halving exchanges: at xor offset 16 >> q the lanes with that bit set
  // keep the upper half of their values; the lane's column index gathers
  // those bits
  int col = 0;
  double b[NK];
#pragma unroll
  for (int u = 0; u < NK; ++u) b[u] = acc[u];
  int n = NK, off = 16;
#pragma unroll
  for (; n > 1; n >>= 1, off >>= 1) {
    const bool hi = lane & off;
#pragma unroll
    for (int u = 0; u < NK / 2; ++u)
      if (u < n / 2) {
        const double send = hi ? b[u] : b[u + n / 2];
        const double keep = hi ? b[u + n / 2] : b[u];
        b[u] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    col = 2 * col + (hi ? 1 : 0);
  }
  double t = b[0];
#pragma unroll
  for (; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  constexpr int LOG = NK == 1 ? 0 : NK == 2 ? 1 : NK == 4 ? 2 : 3;
  if ((lane & ((32 >> LOG) - 1)) == 0) red[warp][col] = t;
  __syncthreads();
  if (threadIdx.x < nk) {
    double sum = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) sum += red[q][threadIdx.x];
    partial[(int64_t)c * ldp + k0 + threadIdx.x] = sum;
  }
}
cudaError_t multidot_partial(int nchunks, const int64_t* cbeg, const int64_t* cend, int ncols, const double* V,
                             int64_t ldv, const double* w, double* partial, int ldp, cudaStream_t st) {
  if (nchunks == 0 || ncols == 0) return cudaSuccess;
  const int nk = ncols >= 8 ? 8 : ncols > 4 ? 8 : ncols > 2 ? 4 : ncols;
  const dim3 grid((unsigned)nchunks, (unsigned)((ncols + nk - 1) / nk));
  switch (nk) {
    case 1: SD_LAUNCH((k_multidot<1>), grid, kRedThreads, 0, st, cbeg, cend, ncols, V, ldv, w, partial, ldp); break;
    case 2: SD_LAUNCH((k_multidot<2>), grid, kRedThreads, 0, st, cbeg, cend, ncols, V, ldv, w, partial, ldp); break;
    case 4: SD_LAUNCH((k_multidot<4>), grid, kRedThreads, 0, st, cbeg, cend, ncols, V, ldv, w, partial, ldp); break;
    default: SD_LAUNCH((k_multidot<8>), grid, kRedThreads, 0, st, cbeg, cend, ncols, V, ldv, w, partial, ldp);
  }
  return cudaGetLastError();
}

// One warp per (segment, column): lane l sums chunks l, l+32, ... of the
// segment in order, then a fixed shuffle tree combines the lanes.
__global__ void __launch_bounds__(128) k_multidot_finish(int nseg, const int* __restrict__ sc_beg,
                                                         const int* __restrict__ sc_end, int ncols,
                                                         const double* __restrict__ partial, int ldp,
                                                         double* __restrict__ h, int ldh, int accumulate) {
  pdl_enter();
  const int idx = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (idx >= nseg * ncols) return;
  const int s = idx / ncols, k = idx - s * ncols;
  double v = 0.0;
  for (int c = sc_beg[s] + lane; c < sc_end[s]; c += 32) v += partial[(int64_t)c * ldp + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) {
    if (accumulate) h[s * ldh + k] += v;
    else h[s * ldh + k] = v;
  }
}
cudaError_t multidot_finish(int nseg, const int* sc_beg, const int* sc_end, int ncols, const double* partial,
                            int ldp, double* h, int ldh, int accumulate, cudaStream_t st) {
  const int tot = nseg * ncols;
  if (tot == 0) return cudaSuccess;
  SD_LAUNCH(k_multidot_finish, (tot + 3) / 4, 128, 0, st, nseg, sc_beg, sc_end, ncols, partial, ldp, h, ldh, accumulate);
  return cudaGetLastError();
}

// grid: nchunks.  w[row] += sign * sum_k coef[seg*ldh + k] * V_k[row]:
// two rows per thread per step, the columns' loads issued eight at a time
// for both rows (sixteen in flight); one DFMA per loaded element.
__global__ void __launch_bounds__(kRedThreads, 4) k_multiaxpy(const int64_t* __restrict__ cbeg,
    const int64_t* __restrict__ cend, const int* __restrict__ cseg, int ncols, const double* __restrict__ V,
    int64_t ldv, const double* __restrict__ coef, int ldh, double sign, double* __restrict__ w) {
  pdl_enter();
  __shared__ double cf[kMaxAxpyCols];
  const int c = blockIdx.x;
  for (int k = threadIdx.x; k < ncols; k += kRedThreads) cf[k] = coef[cseg[c] * ldh + k];
  __syncthreads();
  const int64_t ce = cend[c];
  for (int64_t r = cbeg[c] + threadIdx.x; r < ce; r += 2 * kRedThreads) {
    const int64_t r2 = r + kRedThreads;
    const bool has2 = r2 < ce;
    double s1 = 0.0, s2 = 0.0;
    for (int k0 = 0; k0 < ncols; k0 += 8) {
      double v1[8], v2[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        v1[u] = k0 + u < ncols ? V[(int64_t)(k0 + u) * ldv + r] : 0.0;
        v2[u] = k0 + u < ncols && has2 ? V[(int64_t)(k0 + u) * ldv + r2] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k0 + u < ncols) {
          s1 = fma(cf[k0 + u], v1[u], s1);
          s2 = fma(cf[k0 + u], v2[u], s2);
        }
    }
    w[r] += sign * s1;
    if (has2) w[r2] += sign * s2;
  }
}
cudaError_t multiaxpy(int nchunks, const int64_t* cbeg, const int64_t* cend, const int* cseg, int ncols,
                      const double* V, int64_t ldv, const double* coef, int ldh, double sign, double* w,
                      cudaStream_t st) {
  if (nchunks == 0 || ncols == 0) return cudaSuccess;
  if (ncols > kMaxAxpyCols) return cudaErrorInvalidValue;
  SD_LAUNCH(k_multiaxpy, (unsigned)nchunks, kRedThreads, 0, st, cbeg, cend, cseg, ncols, V, ldv, coef, ldh, sign, w);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(kRedThreads) k_seg_scale(const int64_t* __restrict__ cbeg,
    const int64_t* __restrict__ cend, const int* __restrict__ cseg, const double* __restrict__ in,
    double* __restrict__ out, const double* __restrict__ den, int ldd, int kd, const int* __restrict__ active,
    int sqrt_den) {
  pdl_enter();
  const int c = blockIdx.x;
  const int s = cseg[c];
  double d = den[s * ldd + kd];
  if (sqrt_den) d = sqrt(d);
  const double f = (active[s] && d > 0.0) ? 1.0 / d : 0.0;
  for (int64_t r = cbeg[c] + threadIdx.x; r < cend[c]; r += kRedThreads) out[r] = in[r] * f;
}
cudaError_t seg_scale(int nchunks, const int64_t* cbeg, const int64_t* cend, const int* cseg, const double* in,
                      double* out, const double* den, int ldd, int kd, const int* active, int sqrt_den,
                      cudaStream_t st) {
  if (nchunks == 0) return cudaSuccess;
  SD_LAUNCH(k_seg_scale, nchunks, kRedThreads, 0, st, cbeg, cend, cseg, in, out, den, ldd, kd, active, sqrt_den);
  return cudaGetLastError();
}

}  // namespace sd
