// Krylov-wrapped relaxation (Sec. 3.3.1): on a level, k steps of flexible
// GMRES on K e = b - K x from e = 0, right-preconditioned by one undamped
// additive Vanka sweep per step, then x += Z y with y minimising
// ||beta e1 - H y||.  These kernels hold its vector and scalar parts; the
// sweeps and products are the level's Vanka and SpMV kernels.
//
// The Arnoldi vectors are kept unnormalised (u_0 = r, u_{j+1} = K z_j minus
// its projections), which saves a scaling pass per step: with
// c_ij = (K z_j, u_i) and n_i = ||u_i||^2, the normalised Hessenberg matrix
// is H_ij = c_ij / sqrt(n_i n_j) (i <= j), H_{j+1,j} = sqrt(n_{j+1} / n_j),
// beta = sqrt(n_0), and x += sum_j (y_j / sqrt(n_j)) z_j.
//
// Rows are cut into chunks that never straddle an instance; a reduction's
// last chunk block of an instance (found with a per-instance counter) adds
// that instance's chunk partials in a fixed order, so results are
// deterministic and need no second launch; each instance keeps its own
// scalars.  Scalars of an instance (FP64, stride lds): n_0 at 0, then for
// step j at 1 + j (k+1): c_0j .. c_jj, then n_{j+1}; then the k
// coefficients of the z_j (solved once by the last orthogonalisation).
#include <cmath>

#include "common.cuh"

namespace sd {

constexpr int kKrThreads = 256;

__device__ __forceinline__ int kr_nidx(int i, int k) { return i == 0 ? 0 : 1 + (i - 1) * (k + 1) + i; }

// Last-block completion of a chunked reduction: every block stores its
// partials; the block that finishes last for its instance sums the
// instance's partials (thread t takes chunks t, t+256, ... in order, then a
// fixed block tree) into S and resets the counter.  Returns true in the
// completing block.
template <int NV>
__device__ __forceinline__ bool kr_complete(const KrChunks& ch, int c, int nv, const double (&bsum)[NV],
                                            double* __restrict__ partial, int ldp, int* __restrict__ cnt,
                                            double* __restrict__ S, int lds, const int* __restrict__ cols) {
  __shared__ int last;
  __shared__ double red[kKrThreads / 32];
  const int s = ch.seg[c];
  if (threadIdx.x == 0) {
    for (int i = 0; i < nv; ++i) partial[(int64_t)c * ldp + i] = bsum[i];
    __threadfence();
    const int done = atomicAdd(cnt + s, 1);
    last = done == ch.send[s] - ch.sbeg[s] - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = 0; i < nv; ++i) {
    double v = 0.0;
#pragma unroll 4
    for (int q = ch.sbeg[s] + threadIdx.x; q < ch.send[s]; q += kKrThreads) v += __ldcg(partial + (int64_t)q * ldp + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < kKrThreads / 32; ++q) t += red[q];
      S[(int64_t)s * lds + cols[i]] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) cnt[s] = 0;
  return true;
}

template <int NV>
__device__ __forceinline__ void kr_block_sums(const double (&v)[NV], int nv, double (&out)[NV]) {
  __shared__ double red[kKrThreads / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double t = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) red[warp][i] = t;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = 0.0;
    if (i < nv)
      for (int q = 0; q < kKrThreads / 32; ++q) s += red[q][i];
    out[i] = s;
  }
}

// S[inst][cols[i]] = sum over the instance's rows of A_i[row] * B[row]
// (i < nv, A_i = A + i*lda); copy, when given, receives B.
template <typename T, int NV>
__global__ void __launch_bounds__(kKrThreads) k_kdot(KrChunks ch, int nv, const T* __restrict__ A, int64_t lda,
    const T* __restrict__ B, T* __restrict__ copy, double* __restrict__ partial, int ldp, int* __restrict__ cnt,
    double* __restrict__ S, int lds, KrCols cols) {
  pdl_enter();
  const int c = blockIdx.x;
  T acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = T(0);
  for (int64_t r = ch.beg[c] + threadIdx.x; r < ch.end[c]; r += kKrThreads) {
    const T bv = B[r];
    if (copy) copy[r] = bv;
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nv) acc[i] += A[(int64_t)i * lda + r] * bv;
  }
  double v[NV], bs[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = (double)acc[i];
  kr_block_sums<NV>(v, nv, bs);
  kr_complete<NV>(ch, c, nv, bs, partial, ldp, cnt, S, lds, cols.c);
}

// Least squares min ||beta e1 - H y|| by Givens rotations from the scalars
// (a zero pivot, an exact breakdown or a zero residual, gives y_j = 0);
// returns the coefficients of the unnormalised z_j.
__device__ void kr_solve(const double* __restrict__ q, int k, double* __restrict__ coef) {
  double R[kKrMaxSteps + 1][kKrMaxSteps], g[kKrMaxSteps + 1], nrm[kKrMaxSteps + 1];
  for (int i = 0; i <= k; ++i) nrm[i] = sqrt(fmax(q[kr_nidx(i, k)], 0.0));
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i <= j; ++i) {
      const double d = nrm[i] * nrm[j];
      R[i][j] = d > 0.0 ? q[1 + j * (k + 1) + i] / d : 0.0;
    }
    R[j + 1][j] = nrm[j] > 0.0 ? nrm[j + 1] / nrm[j] : 0.0;
  }
  g[0] = nrm[0];
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
  for (int j = 0; j < k; ++j) coef[j] = nrm[j] > 0.0 ? y[j] / nrm[j] : 0.0;
}

// Step j: W -= sum_{i<=j} (c_ij / n_i) U_i, then n_{j+1} = ||W||^2.
template <typename T>
__global__ void __launch_bounds__(kKrThreads) k_kaxpy_norm(KrChunks ch, int j, int k, const T* __restrict__ U,
    int64_t ldu, T* __restrict__ W, double* __restrict__ partial, int ldp, int* __restrict__ cnt,
    double* __restrict__ S, int lds) {
  pdl_enter();
  __shared__ T cf[kKrMaxSteps];
  const int c = blockIdx.x;
  const double* q = S + (int64_t)ch.seg[c] * lds;
  if (threadIdx.x <= j) {
    const double n = q[kr_nidx(threadIdx.x, k)];
    cf[threadIdx.x] = n > 0.0 ? T(q[1 + j * (k + 1) + threadIdx.x] / n) : T(0);
  }
  __syncthreads();
  T acc = T(0);
  for (int64_t r = ch.beg[c] + threadIdx.x; r < ch.end[c]; r += kKrThreads) {
    T s = T(0);
    for (int i = 0; i <= j; ++i) s += cf[i] * U[(int64_t)i * ldu + r];
    const T wn = W[r] - s;
    W[r] = wn;
    acc += wn * wn;
  }
  double v[1] = {(double)acc}, bs[1];
  kr_block_sums<1>(v, 1, bs);
  KrCols col;
  col.c[0] = kr_nidx(j + 1, k);
  const bool done = kr_complete<1>(ch, c, 1, bs, partial, ldp, cnt, S, lds, col.c);
  // after the last step, the completing block solves the least-squares
  // problem of its instance once and stores the coefficients of the z_j
  if (done && j + 1 == k && threadIdx.x == 0) {
    double* qs = S + (int64_t)ch.seg[c] * lds;
    double coef[kKrMaxSteps];
    kr_solve(qs, k, coef);
    for (int jj = 0; jj < k; ++jj) qs[1 + k * (k + 1) + jj] = coef[jj];
  }
}

// x = (set ? 0 : x) + sum_j coef_j Z_j with the coefficients the last
// orthogonalisation stored; optionally the FP64 copy x64 and the level-0
// cycle output out64 = dir ? r64 : x.
template <typename T>
__global__ void __launch_bounds__(kKrThreads) k_kupdate(KrChunks ch, int k, const T* __restrict__ Z, int64_t ldz,
    const double* __restrict__ S, int lds, T* __restrict__ x, int set, double* __restrict__ x64,
    const uint8_t* __restrict__ dir, const double* __restrict__ r64, double* __restrict__ out64) {
  pdl_enter();
  __shared__ T y[kKrMaxSteps];
  const int c = blockIdx.x;
  if (threadIdx.x < k) y[threadIdx.x] = T(S[(int64_t)ch.seg[c] * lds + 1 + k * (k + 1) + threadIdx.x]);
  __syncthreads();
  for (int64_t r = ch.beg[c] + threadIdx.x; r < ch.end[c]; r += kKrThreads) {
    T v = set ? T(0) : x[r];
    for (int j = 0; j < k; ++j) v += y[j] * Z[(int64_t)j * ldz + r];
    x[r] = v;
    if (x64) x64[r] = (double)v;
    if (out64) out64[r] = dir[r] ? r64[r] : (double)v;
  }
}

// ------------------------------------------------------------- launchers
template <typename T>
cudaError_t kr_norm0(const KrChunks& ch, const T* r, T* u0, double* partial, int ldp, int* cnt, double* S, int lds,
                     cudaStream_t st) {
  if (ch.n == 0) return cudaSuccess;
  KrCols cols;
  cols.c[0] = 0;
  SD_LAUNCH((k_kdot<T, 1>), ch.n, kKrThreads, 0, st, ch, 1, r, 0, r, u0 == r ? nullptr : u0, partial, ldp, cnt, S, lds, cols);
  return cudaGetLastError();
}

template <typename T>
cudaError_t kr_project(const KrChunks& ch, int j, int k, const T* U, int64_t ldu, const T* w, double* partial,
                       int ldp, int* cnt, double* S, int lds, cudaStream_t st) {
  if (ch.n == 0) return cudaSuccess;
  if (j >= kKrMaxSteps || k > kKrMaxSteps) return cudaErrorInvalidValue;
  KrCols cols;
  for (int i = 0; i <= j; ++i) cols.c[i] = 1 + j * (k + 1) + i;
  SD_LAUNCH((k_kdot<T, kKrMaxSteps>), ch.n, kKrThreads, 0, st, ch, j + 1, U, ldu, w, (T*)nullptr, partial, ldp, cnt, S, lds,
                                                      cols);
  return cudaGetLastError();
}

template <typename T>
cudaError_t kr_orthogonalise(const KrChunks& ch, int j, int k, const T* U, int64_t ldu, T* w, double* partial,
                             int ldp, int* cnt, double* S, int lds, cudaStream_t st) {
  if (ch.n == 0) return cudaSuccess;
  if (j >= kKrMaxSteps || k > kKrMaxSteps) return cudaErrorInvalidValue;
  SD_LAUNCH((k_kaxpy_norm<T>), ch.n, kKrThreads, 0, st, ch, j, k, U, ldu, w, partial, ldp, cnt, S, lds);
  return cudaGetLastError();
}

template <typename T>
cudaError_t kr_update(const KrChunks& ch, int k, const T* Z, int64_t ldz, const double* S, int lds, T* x, int set,
                      double* x64, const uint8_t* dir, const double* r64, double* out64, cudaStream_t st) {
  if (ch.n == 0) return cudaSuccess;
  if (k > kKrMaxSteps) return cudaErrorInvalidValue;
  SD_LAUNCH((k_kupdate<T>), ch.n, kKrThreads, 0, st, ch, k, Z, ldz, S, lds, x, set, x64, dir, r64, out64);
  return cudaGetLastError();
}

#define SD_KR(T)                                                                                                   \
  template cudaError_t kr_norm0<T>(const KrChunks&, const T*, T*, double*, int, int*, double*, int, cudaStream_t); \
  template cudaError_t kr_project<T>(const KrChunks&, int, int, const T*, int64_t, const T*, double*, int, int*,  \
                                     double*, int, cudaStream_t);                                                \
  template cudaError_t kr_orthogonalise<T>(const KrChunks&, int, int, const T*, int64_t, T*, double*, int, int*,  \
                                           double*, int, cudaStream_t);                                          \
  template cudaError_t kr_update<T>(const KrChunks&, int, const T*, int64_t, const double*, int, T*, int, double*, \
                                    const uint8_t*, const double*, double*, cudaStream_t);
SD_KR(float)
SD_KR(double)
#undef SD_KR

}  // namespace sd
