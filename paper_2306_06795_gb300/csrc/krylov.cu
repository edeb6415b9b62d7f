// Krylov-wrapped relaxation (Sec. 3.3.1): on a level, k steps of flexible
// GMRES on K e = b - K x from e = 0, right-preconditioned by one undamped
// additive Vanka sweep per step, then x += Z y with y minimising
// ||beta e1 - H y||.  These kernels hold its vector and scalar parts; the
// sweeps and products are the level's Vanka and SpMV kernels.  Rows are cut
// into chunks that never straddle an instance, and every reduction sums the
// chunk partials of an instance in a fixed order, so results are
// deterministic; each instance keeps its own scalars.
//
// Scalars of an instance (FP64, stride lds): [0] = ||r||^2, then column j
// of H at 1 + j (k+1) + i (i <= j: projections, i = j+1: the squared norm
// of the orthogonalised vector), then y at 1 + k (k+1) + j.
#include <cmath>

#include "common.cuh"

namespace sd {

constexpr int kKrThreads = 256;

// partial[c*ldp + i] = sum over chunk c of A_i[row] * B[row], i < nv
// (A_i = A + i*lda); per-thread sums in T, warp and block sums in FP64.
template <typename T, int NV>
__global__ void __launch_bounds__(kKrThreads) k_kdot(const int64_t* __restrict__ cbeg,
    const int64_t* __restrict__ cend, int nv, const T* __restrict__ A, int64_t lda, const T* __restrict__ B,
    double* __restrict__ partial, int ldp) {
  __shared__ double red[kKrThreads / 32][NV];
  const int c = blockIdx.x;
  T acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = T(0);
  for (int64_t r = cbeg[c] + threadIdx.x; r < cend[c]; r += kKrThreads) {
    const T bv = B[r];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nv) acc[i] += A[(int64_t)i * lda + r] * bv;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double v = (double)acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][i] = v;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double s = 0.0;
    for (int q = 0; q < kKrThreads / 32; ++q) s += red[q][threadIdx.x];
    partial[(int64_t)c * ldp + threadIdx.x] = s;
  }
}

// W[row] -= sum_{i<nv} coef_i A_i[row] (coef of the row's instance at
// S[inst*lds + c0 + i]), then partial[c*ldp] = sum over chunk c of W^2.
template <typename T>
__global__ void __launch_bounds__(kKrThreads) k_kaxpy_norm(const int64_t* __restrict__ cbeg,
    const int64_t* __restrict__ cend, const int* __restrict__ cseg, int nv, const T* __restrict__ A, int64_t lda,
    const double* __restrict__ S, int lds, int c0, T* __restrict__ W, double* __restrict__ partial, int ldp) {
  __shared__ double red[kKrThreads / 32];
  __shared__ T cf[kKrMaxSteps + 1];
  const int c = blockIdx.x;
  if (threadIdx.x < nv) cf[threadIdx.x] = T(S[(int64_t)cseg[c] * lds + c0 + threadIdx.x]);
  __syncthreads();
  T acc = T(0);
  for (int64_t r = cbeg[c] + threadIdx.x; r < cend[c]; r += kKrThreads) {
    T s = T(0);
    for (int i = 0; i < nv; ++i) s += cf[i] * A[(int64_t)i * lda + r];
    const T wn = W[r] - s;
    W[r] = wn;
    acc += wn * wn;
  }
  double v = (double)acc;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kKrThreads / 32; ++q) s += red[q];
    partial[(int64_t)c * ldp] = s;
  }
}

// One warp per (instance, column): S[inst*lds + o + col] = sum of the
// instance's chunk partials in chunk order.
__global__ void __launch_bounds__(128) k_kfinish(int ninst, const int* __restrict__ sc_beg,
    const int* __restrict__ sc_end, int ncols, const double* __restrict__ partial, int ldp, double* __restrict__ S,
    int lds, int o) {
  const int idx = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (idx >= ninst * ncols) return;
  const int s = idx / ncols, k = idx - s * ncols;
  double v = 0.0;
  for (int c = sc_beg[s] + lane; c < sc_end[s]; c += 32) v += partial[(int64_t)c * ldp + k];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if (lane == 0) S[(int64_t)s * lds + o + k] = v;
}

// out[row] = in[row] / sqrt(S[inst*lds + o]) (0 when that squared norm is 0)
template <typename T>
__global__ void __launch_bounds__(kKrThreads) k_kscale(const int64_t* __restrict__ cbeg,
    const int64_t* __restrict__ cend, const int* __restrict__ cseg, const T* __restrict__ in, T* __restrict__ out,
    const double* __restrict__ S, int lds, int o) {
  const int c = blockIdx.x;
  const double n2 = S[(int64_t)cseg[c] * lds + o];
  const T f = n2 > 0.0 ? T(1.0 / sqrt(n2)) : T(0);
  for (int64_t r = cbeg[c] + threadIdx.x; r < cend[c]; r += kKrThreads) out[r] = in[r] * f;
}

// Least squares min ||beta e1 - H y|| per instance by Givens rotations;
// a zero pivot (exact breakdown, or a zero residual) gives y_j = 0.
__global__ void k_kls(int ninst, int k, double* __restrict__ S, int lds) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= ninst) return;
  double* q = S + (size_t)s * lds;
  double R[kKrMaxSteps + 1][kKrMaxSteps], g[kKrMaxSteps + 1];
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i <= j; ++i) R[i][j] = q[1 + j * (k + 1) + i];
    R[j + 1][j] = sqrt(fmax(q[1 + j * (k + 1) + j + 1], 0.0));
  }
  g[0] = sqrt(fmax(q[0], 0.0));
  for (int i = 1; i <= k; ++i) g[i] = 0.0;
  for (int j = 0; j < k; ++j) {
    const double a = R[j][j], b = R[j + 1][j];
    const double den = hypot(a, b);
    const double cs = den > 0.0 ? a / den : 1.0, sn = den > 0.0 ? b / den : 0.0;
    for (int jj = j; jj < k; ++jj) {
      const double t = cs * R[j][jj] + sn * R[j + 1][jj];
      R[j + 1][jj] = -sn * R[j][jj] + cs * R[j + 1][jj];
      R[j][jj] = t;
    }
    const double t = cs * g[j] + sn * g[j + 1];
    g[j + 1] = -sn * g[j] + cs * g[j + 1];
    g[j] = t;
  }
  double y[kKrMaxSteps];
  for (int j = k - 1; j >= 0; --j) {
    double v = g[j];
    for (int jj = j + 1; jj < k; ++jj) v -= R[j][jj] * y[jj];
    y[j] = R[j][j] != 0.0 ? v / R[j][j] : 0.0;
  }
  for (int j = 0; j < k; ++j) q[1 + k * (k + 1) + j] = y[j];
}

// x[row] = (set ? 0 : x[row]) + sum_j y_j Z_j[row]; optionally the FP64
// copy x64 and the level-0 cycle output out64 = dir ? r64 : x.
template <typename T>
__global__ void __launch_bounds__(kKrThreads) k_kupdate(const int64_t* __restrict__ cbeg,
    const int64_t* __restrict__ cend, const int* __restrict__ cseg, int k, const T* __restrict__ Z, int64_t ldz,
    const double* __restrict__ S, int lds, int oy, T* __restrict__ x, int set, double* __restrict__ x64,
    const uint8_t* __restrict__ dir, const double* __restrict__ r64, double* __restrict__ out64) {
  __shared__ T y[kKrMaxSteps];
  const int c = blockIdx.x;
  if (threadIdx.x < k) y[threadIdx.x] = T(S[(int64_t)cseg[c] * lds + oy + threadIdx.x]);
  __syncthreads();
  for (int64_t r = cbeg[c] + threadIdx.x; r < cend[c]; r += kKrThreads) {
    T v = set ? T(0) : x[r];
    for (int j = 0; j < k; ++j) v += y[j] * Z[(int64_t)j * ldz + r];
    x[r] = v;
    if (x64) x64[r] = (double)v;
    if (out64) out64[r] = dir[r] ? r64[r] : (double)v;
  }
}

// ------------------------------------------------------------- launchers
template <typename T>
cudaError_t kr_dot(const KrChunks& ch, int nv, const T* A, int64_t lda, const T* B, double* partial, int ldp,
                   double* S, int lds, int o, int ninst, cudaStream_t st) {
  if (ch.n == 0 || nv == 0) return cudaSuccess;
  if (nv > kKrMaxSteps + 1) return cudaErrorInvalidValue;
  if (nv == 1)
    k_kdot<T, 1><<<ch.n, kKrThreads, 0, st>>>(ch.beg, ch.end, nv, A, lda, B, partial, ldp);
  else
    k_kdot<T, kKrMaxSteps + 1><<<ch.n, kKrThreads, 0, st>>>(ch.beg, ch.end, nv, A, lda, B, partial, ldp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_kfinish<<<(ninst * nv + 3) / 4, 128, 0, st>>>(ninst, ch.sbeg, ch.send, nv, partial, ldp, S, lds, o);
  return cudaGetLastError();
}

template <typename T>
cudaError_t kr_axpy_norm(const KrChunks& ch, int nv, const T* A, int64_t lda, int c0, T* W, double* partial, int ldp,
                         double* S, int lds, int o, int ninst, cudaStream_t st) {
  if (ch.n == 0) return cudaSuccess;
  if (nv > kKrMaxSteps + 1) return cudaErrorInvalidValue;
  k_kaxpy_norm<T><<<ch.n, kKrThreads, 0, st>>>(ch.beg, ch.end, ch.seg, nv, A, lda, S, lds, c0, W, partial, ldp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_kfinish<<<(ninst + 3) / 4, 128, 0, st>>>(ninst, ch.sbeg, ch.send, 1, partial, ldp, S, lds, o);
  return cudaGetLastError();
}

template <typename T>
cudaError_t kr_scale(const KrChunks& ch, const T* in, T* out, const double* S, int lds, int o, cudaStream_t st) {
  if (ch.n == 0) return cudaSuccess;
  k_kscale<T><<<ch.n, kKrThreads, 0, st>>>(ch.beg, ch.end, ch.seg, in, out, S, lds, o);
  return cudaGetLastError();
}

cudaError_t kr_ls(int ninst, int k, double* S, int lds, cudaStream_t st) {
  if (k > kKrMaxSteps) return cudaErrorInvalidValue;
  k_kls<<<(ninst + 63) / 64, 64, 0, st>>>(ninst, k, S, lds);
  return cudaGetLastError();
}

template <typename T>
cudaError_t kr_update(const KrChunks& ch, int k, const T* Z, int64_t ldz, const double* S, int lds, int oy, T* x,
                      int set, double* x64, const uint8_t* dir, const double* r64, double* out64, cudaStream_t st) {
  if (ch.n == 0) return cudaSuccess;
  k_kupdate<T><<<ch.n, kKrThreads, 0, st>>>(ch.beg, ch.end, ch.seg, k, Z, ldz, S, lds, oy, x, set, x64, dir, r64,
                                            out64);
  return cudaGetLastError();
}

#define SD_KR(T)                                                                                              \
  template cudaError_t kr_dot<T>(const KrChunks&, int, const T*, int64_t, const T*, double*, int, double*, int, \
                                 int, int, cudaStream_t);                                                      \
  template cudaError_t kr_axpy_norm<T>(const KrChunks&, int, const T*, int64_t, int, T*, double*, int, double*, \
                                       int, int, int, cudaStream_t);                                           \
  template cudaError_t kr_scale<T>(const KrChunks&, const T*, T*, const double*, int, int, cudaStream_t);        \
  template cudaError_t kr_update<T>(const KrChunks&, int, const T*, int64_t, const double*, int, int, T*, int,  \
                                    double*, const uint8_t*, const double*, double*, cudaStream_t);
SD_KR(float)
SD_KR(double)
#undef SD_KR

}  // namespace sd
