// Device-side bookkeeping of restarted FGMRES (Sec. 4): per instance, the
// Hessenberg column, Givens rotations, the residual estimate, the running
// flag and the scale of the next Krylov vector are updated on the device,
// so an Arnoldi step needs no host round trip.  All arithmetic of an
// instance runs in a fixed order.
#include <cmath>

#include "common.cuh"

namespace sd {


// Start of a restart cycle: h[s*ldh] = ||r_s||^2.
__global__ void __launch_bounds__(256) k_fg_start(int ninst, int m, FgState st, const double* __restrict__ h, int ldh, double rtol, int maxit,
                           int first) {
  pdl_enter();
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < ninst; s += blockDim.x) {
    const double beta = sqrt(h[s * ldh]);
    if (first) st.bnorm[s] = beta;  // the first residual is b itself (x0 = 0) or b - K0 x0
    if (!isfinite(beta)) atomicOr(st.err, 1);
    const double bn = st.bnorm[s];
    const bool done = bn == 0.0 || beta <= rtol * bn;
    const bool run = !done && st.its[s] < maxit && isfinite(beta);
    st.run[s] = run;
    st.kcol[s] = 0;
    double* g = st.g + (size_t)s * (m + 1);
    for (int i = 0; i <= m; ++i) g[i] = 0.0;
    g[0] = beta;
    st.scale[s] = run ? 1.0 / beta : 0.0;
    if (run) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) st.stat[m] = any;
}

// Givens update of Arnoldi column j of instance s, run by all threads of one
// block: col[i] = h1[i] + h2[i] (the two Gram-Schmidt passes), col[j+1] =
// ||w|| = sqrt(hn2); the previous rotations are applied in order by thread 0,
// the new rotation zeroes col[j+1], the residual estimate |g[j+1]| decides
// whether the instance keeps running, and the running flag is OR-ed into
// stat[j] (zeroed beforehand).  Shared scratch: col[j+2], csS[j], snS[j],
// wmax[blockDim.x / 32].
__device__ void fg_column_update(int s, int m, int j, const FgState& st, const double* __restrict__ h1,
                                 const double* __restrict__ h2, double hn2, double rtol, int maxit, double* col,
                                 double* csS, double* snS, double* wmax) {
  if (!st.run[s]) {  // block-uniform
    if (threadIdx.x == 0) st.scale[s] = 0.0;
    return;
  }
  double* H = st.H + (size_t)s * (m + 1) * m;
  double* cs = st.cs + (size_t)s * m;
  double* sn = st.sn + (size_t)s * m;
  double hm = 0.0;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    col[i] = h1[i] + h2[i];
    hm = fmax(hm, fabs(col[i]));
  }
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    csS[i] = cs[i];
    snS[i] = sn[i];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) hm = fmax(hm, __shfl_xor_sync(0xffffffffu, hm, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = hm;
  __syncthreads();
  if (threadIdx.x == 0) {
    double hmax = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) hmax = fmax(hmax, wmax[q]);
    double* g = st.g + (size_t)s * (m + 1);
    const double hn = sqrt(hn2);
    col[j + 1] = hn;
    const bool breakdown = !(hn > 1e-14 * fmax(hmax, 1e-300));
    for (int i = 0; i < j; ++i) {
      const double t = csS[i] * col[i] + snS[i] * col[i + 1];
      col[i + 1] = -snS[i] * col[i] + csS[i] * col[i + 1];
      col[i] = t;
    }
    const double den = hypot(col[j], col[j + 1]);
    // den == 0: the rotated column vanishes (K0 z_j lies in span V_{j-1}
    // and adds nothing); column j is left out of the least-squares solve
    // and the instance stops as at a breakdown
    const bool degenerate = !(den > 0.0);
    const double c = degenerate ? 1.0 : col[j] / den, sj = degenerate ? 0.0 : col[j + 1] / den;
    cs[j] = c;
    sn[j] = sj;
    col[j] = den;
    col[j + 1] = 0.0;
    const double gj = g[j];
    g[j + 1] = -sj * gj;
    g[j] = c * gj;
    st.its[s] += 1;
    st.kcol[s] = degenerate ? j : j + 1;
    if (!isfinite(g[j + 1])) atomicOr(st.err, 1);
    const bool run = !(fabs(g[j + 1]) <= rtol * st.bnorm[s]) && !breakdown && !degenerate && st.its[s] < maxit &&
                     j + 1 < m && isfinite(g[j + 1]);
    st.run[s] = run;
    st.scale[s] = run ? 1.0 / hn : 0.0;
    if (run) atomicOr(st.stat + j, 1);
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) H[i * m + j] = col[i];
}

// Arnoldi step j (any restart length): h1buf[s*ldh + i] and h2buf hold the
// two Gram-Schmidt passes, ||w||^2 in h1buf[s*ldh + j + 1].  One block per
// instance.
__global__ void __launch_bounds__(64) k_fg_update(int ninst, int m, int j, FgState st, const double* __restrict__ h1buf,
                            const double* __restrict__ h2buf, int ldh, double rtol, int maxit) {
  griddep_wait();
  extern __shared__ double fsm[];
  double* col = fsm;            // [j+2]
  double* csS = col + (m + 2);  // [j]
  double* snS = csS + m;        // [j]
  __shared__ double wmax[2];
  const int s = blockIdx.x;
  if (s >= ninst) return;
  const double* h1 = h1buf + (size_t)s * ldh;
  fg_column_update(s, m, j, st, h1, h2buf + (size_t)s * ldh, h1[j + 1], rtol, maxit, col, csS, snS, wmax);
}

// ------------------------------------------------ fused Arnoldi passes
// Classical Gram-Schmidt twice for up to kArMaxCols Krylov columns, in
// three launches over 2048-row chunks that never straddle an instance:
//   k_ar_dots:        h1 = V^T w
//   k_ar_axpy_dots:   w -= V h1, then h2 = V^T w (each row's V entries are
//                     read again right after, from L1)
//   k_ar_axpy_norm:   w -= V h2, ||w||^2, and the Givens update of the
//                     instance (fg_column_update)
// NK, the number of columns, is a template parameter, so that every
// accumulator and every loaded entry lives in registers and no DFMA is
// spent on absent columns: GB300's FP64 rate, not HBM, bounds these passes
// (one DFMA per loaded element).  Each block reduces its chunk with a
// transposed butterfly and adds its warps in order; the last block of an
// instance (per-instance counter) adds the instance's chunk partials in
// chunk order: deterministic, one launch per reduction.
constexpr int kArThreads = 256;

template <int NK>
__device__ __forceinline__ void ar_block_sums(const double (&acc)[NK], double* red, double* bsum) {
  constexpr int NP = NK <= 1 ? 1 : NK <= 2 ? 2 : NK <= 4 ? 4 : NK <= 8 ? 8 : NK <= 16 ? 16 : 32;
  constexpr int LOG = NP == 1 ? 0 : NP == 2 ? 1 : NP == 4 ? 2 : NP == 8 ? 3 : NP == 16 ? 4 : 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double b[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) b[k] = k < NK ? acc[k] : 0.0;
  // halving exchanges: at xor offset 16 >> q the lanes with that bit set
  // keep the upper half of their values; the lane's column gathers the bits
  int col = 0, off = 16;
#pragma unroll
  for (int nn = NP; nn > 1; nn >>= 1, off >>= 1) {
    const bool hi = lane & off;
#pragma unroll
    for (int u = 0; u < NP / 2; ++u)
      if (u < nn / 2) {
        const double send = hi ? b[u] : b[u + nn / 2];
        const double keep = hi ? b[u + nn / 2] : b[u];
        b[u] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
    col = 2 * col + (hi ? 1 : 0);
  }
  double t = b[0];
#pragma unroll
  for (; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  if ((lane & ((32 >> LOG) - 1)) == 0) red[warp * 32 + col] = t;
  __syncthreads();
  if (threadIdx.x < NK) {
    double v = 0.0;
    for (int q = 0; q < kArThreads / 32; ++q) v += red[q * 32 + threadIdx.x];
    bsum[threadIdx.x] = v;
  }
  __syncthreads();
}

// Writes the chunk's sums, counts the chunk, and in the instance's last
// block sums all its chunk partials in chunk order into tot[0..NK).
template <int NK>
__device__ __forceinline__ bool ar_complete(const KrChunks& ch, int c, const double* bsum, double* __restrict__ partial,
                                            int ldp, int* __restrict__ cnt, double* tot) {
  __shared__ int last;
  const int s = ch.seg[c];
  if (threadIdx.x < NK) {
    partial[(int64_t)c * ldp + threadIdx.x] = bsum[threadIdx.x];
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(cnt + s, 1) == ch.send[s] - ch.sbeg[s] - 1;
  __syncthreads();
  if (!last) return false;
  __threadfence();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = warp; k < NK; k += kArThreads / 32) {
    double v = 0.0;
    for (int q = ch.sbeg[s] + lane; q < ch.send[s]; q += 32) v += __ldcg(partial + (int64_t)q * ldp + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) tot[k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) cnt[s] = 0;
  return true;
}

template <int NK, int U>
__global__ void __launch_bounds__(kArThreads, 2) k_ar_dots(KrChunks ch, const double* __restrict__ V, int64_t ldv,
    const double* __restrict__ w, double* __restrict__ partial, int ldp, int* __restrict__ cnt,
    double* __restrict__ hout, int ldh, int* __restrict__ zero_flag) {
  griddep_wait();
  __shared__ double red[kArThreads];
  __shared__ double bsum[NK], tot[NK];
  const int c = blockIdx.x;
  if (zero_flag && c == 0 && threadIdx.x == 0) *zero_flag = 0;
  double acc[NK];
#pragma unroll
  for (int k = 0; k < NK; ++k) acc[k] = 0.0;
  const int64_t re = ch.end[c];
  for (int64_t r = ch.beg[c] + threadIdx.x; r < re; r += kArThreads * U) {
    double wv[U], v[U][NK];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool ok = r + u * kArThreads < re;
      wv[u] = ok ? w[r + u * kArThreads] : 0.0;
#pragma unroll
      for (int k = 0; k < NK; ++k) v[u][k] = ok ? V[(int64_t)k * ldv + r + u * kArThreads] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < NK; ++k) acc[k] = fma(v[u][k], wv[u], acc[k]);
  }
  ar_block_sums<NK>(acc, red, bsum);
  if (ar_complete<NK>(ch, c, bsum, partial, ldp, cnt, tot) && threadIdx.x < NK)
    hout[(int64_t)ch.seg[c] * ldh + threadIdx.x] = tot[threadIdx.x];
}

template <int NK>
__global__ void __launch_bounds__(kArThreads, 2) k_ar_axpy_dots(KrChunks ch, const double* __restrict__ V, int64_t ldv,
    const double* __restrict__ coef, int ldh, double* __restrict__ w, double* __restrict__ partial, int ldp,
    int* __restrict__ cnt, double* __restrict__ hout) {
  griddep_wait();
  __shared__ double red[kArThreads];
  __shared__ double cf[NK], bsum[NK], tot[NK];
  const int c = blockIdx.x;
  const int s = ch.seg[c];
  if (threadIdx.x < NK) cf[threadIdx.x] = coef[(int64_t)s * ldh + threadIdx.x];
  __syncthreads();
  // the coefficients are read from shared memory at each use (volatile), so
  // that the NK accumulators, not NK hoisted coefficients, hold the registers
  const volatile double* cfv = cf;
  double acc[NK];
#pragma unroll
  for (int k = 0; k < NK; ++k) acc[k] = 0.0;
  constexpr int G = 8;
  const int64_t re = ch.end[c];
  for (int64_t r = ch.beg[c] + threadIdx.x; r < re; r += kArThreads) {
    double t = w[r];
#pragma unroll
    for (int k0 = 0; k0 < NK; k0 += G) {
      double v[G];
#pragma unroll
      for (int k = 0; k < G; ++k) v[k] = k0 + k < NK ? V[(int64_t)(k0 + k) * ldv + r] : 0.0;
#pragma unroll
      for (int k = 0; k < G; ++k)
        if (k0 + k < NK) t = fma(-cfv[k0 + k], v[k], t);
    }
    w[r] = t;
#pragma unroll
    for (int k0 = 0; k0 < NK; k0 += G) {
      double v[G];
#pragma unroll
      for (int k = 0; k < G; ++k) v[k] = k0 + k < NK ? V[(int64_t)(k0 + k) * ldv + r] : 0.0;
#pragma unroll
      for (int k = 0; k < G; ++k)
        if (k0 + k < NK) acc[k0 + k] = fma(v[k], t, acc[k0 + k]);
    }
  }
  ar_block_sums<NK>(acc, red, bsum);
  if (ar_complete<NK>(ch, c, bsum, partial, ldp, cnt, tot) && threadIdx.x < NK)
    hout[(int64_t)s * ldh + threadIdx.x] = tot[threadIdx.x];
}

template <int NK>
__global__ void __launch_bounds__(kArThreads, 2) k_ar_axpy_norm(KrChunks ch, const double* __restrict__ V, int64_t ldv,
    const double* __restrict__ h1buf, const double* __restrict__ h2buf, int ldh, double* __restrict__ w,
    double* __restrict__ partial, int ldp, int* __restrict__ cnt, int m, int j, FgState st, double rtol, int maxit) {
  griddep_wait();
  __shared__ double red[kArThreads];
  __shared__ double cf[NK], bsum[1], tot[1];
  __shared__ double col[NK + 2], csS[NK], snS[NK], wmax[kArThreads / 32];
  const int c = blockIdx.x;
  const int s = ch.seg[c];
  if (threadIdx.x < NK) cf[threadIdx.x] = h2buf[(int64_t)s * ldh + threadIdx.x];
  __syncthreads();
  const volatile double* cfv = cf;  // read at each use, as in k_ar_axpy_dots
  double acc[1] = {0.0};
  // P rows per thread per step with their column loads issued together
  // (the pass reads V once, from DRAM: more loads in flight)
  constexpr int G = 8, P = 4;
  const int64_t re = ch.end[c];
  for (int64_t r = ch.beg[c] + threadIdx.x; r < re; r += kArThreads * P) {
    double t[P];
#pragma unroll
    for (int p = 0; p < P; ++p) t[p] = r + p * kArThreads < re ? w[r + p * kArThreads] : 0.0;
#pragma unroll
    for (int k0 = 0; k0 < NK; k0 += G) {
      double v[P][G];
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int k = 0; k < G; ++k)
          v[p][k] = k0 + k < NK && r + p * kArThreads < re ? V[(int64_t)(k0 + k) * ldv + r + p * kArThreads] : 0.0;
#pragma unroll
      for (int k = 0; k < G; ++k)
        if (k0 + k < NK) {
          const double ck = cfv[k0 + k];
#pragma unroll
          for (int p = 0; p < P; ++p) t[p] = fma(-ck, v[p][k], t[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
      if (r + p * kArThreads < re) {
        w[r + p * kArThreads] = t[p];
        acc[0] = fma(t[p], t[p], acc[0]);
      }
  }
  ar_block_sums<1>(acc, red, bsum);
  if (ar_complete<1>(ch, c, bsum, partial, ldp, cnt, tot))
    fg_column_update(s, m, j, st, h1buf + (int64_t)s * ldh, h2buf + (int64_t)s * ldh, tot[0], rtol, maxit, col, csS,
                     snS, wmax);
}

// y of the least-squares problem by back substitution (per instance).
__global__ void k_fg_solve(int ninst, int m, FgState st, int ldh) {
  pdl_enter();
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ninst; s += gridDim.x * blockDim.x) {
    const int k = st.kcol[s];
    const double* H = st.H + (size_t)s * (m + 1) * m;
    const double* g = st.g + (size_t)s * (m + 1);
    double* y = st.y + (size_t)s * ldh;
    for (int i = 0; i < ldh; ++i) y[i] = 0.0;
    for (int i = k - 1; i >= 0; --i) {
      double v = g[i];
      for (int q = i + 1; q < k; ++q) v -= H[i * m + q] * y[q];
      y[i] = v / H[i * m + i];
    }
  }
}

// out[row] = in[row] * f[seg(row)] (and its FP32 rounding in out32)
__global__ void __launch_bounds__(256) k_seg_mul(const int64_t* __restrict__ cbeg, const int64_t* __restrict__ cend,
                                                 const int* __restrict__ cseg, const double* in, double* out,
                                                 const double* __restrict__ f, float* __restrict__ out32) {
  pdl_enter();
  const int c = blockIdx.x;
  const double v = f[cseg[c]];
  for (int64_t r = cbeg[c] + threadIdx.x; r < cend[c]; r += 256) {
    const double o = v == 0.0 ? 0.0 : in[r] * v;
    out[r] = o;
    if (out32) out32[r] = (float)o;
  }
}

cudaError_t fg_start(int ninst, int m, const FgState& st, const double* h, int ldh, double rtol, int maxit, int first,
                     cudaStream_t s) {
  SD_LAUNCH(k_fg_start, 1, 256, 0, s, ninst, m, st, h, ldh, rtol, maxit, first);
  return cudaGetLastError();
}
#define SD_AR_CASES(X)                                                                                         \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16) X(17) X(18) X(19) X(20) \
  X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)

cudaError_t ar_dots(const KrChunks& ch, int nc, const double* V, int64_t ldv, const double* w, double* partial,
                    int ldp, int* cnt, double* h, int ldh, int* zero_flag, cudaStream_t s) {
  if (ch.n == 0) return cudaSuccess;
  switch (nc) {
#define SD_AR_DOTS(K)                                                                                           \
  case K:                                                                                                      \
    return launch_pdl(k_ar_dots<K, (K <= 8 ? 4 : K <= 16 ? 2 : 1)>, dim3(ch.n), dim3(kArThreads), 0, s, ch, V,   \
                      ldv, w,                                                                                     \
                      partial, ldp, cnt, h, ldh, zero_flag);
    SD_AR_CASES(SD_AR_DOTS)
#undef SD_AR_DOTS
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t ar_axpy_dots(const KrChunks& ch, int nc, const double* V, int64_t ldv, const double* coef, int ldh,
                         double* w, double* partial, int ldp, int* cnt, double* h, cudaStream_t s) {
  if (ch.n == 0) return cudaSuccess;
  switch (nc) {
#define SD_AR_AD(K)                                                                                              \
  case K:                                                                                                       \
    return launch_pdl(k_ar_axpy_dots<K>, dim3(ch.n), dim3(kArThreads), 0, s, ch, V, ldv, coef, ldh, w, partial, \
                      ldp, cnt, h);
    SD_AR_CASES(SD_AR_AD)
#undef SD_AR_AD
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t ar_axpy_norm_update(const KrChunks& ch, int nc, const double* V, int64_t ldv, const double* h1,
                                const double* h2, int ldh, double* w, double* partial, int ldp, int* cnt, int m, int j,
                                const FgState& st, double rtol, int maxit, cudaStream_t s) {
  if (ch.n == 0) return cudaSuccess;
  if (nc != j + 1) return cudaErrorInvalidValue;
  switch (nc) {
#define SD_AR_AN(K)                                                                                              \
  case K:                                                                                                       \
    return launch_pdl(k_ar_axpy_norm<K>, dim3(ch.n), dim3(kArThreads), 0, s, ch, V, ldv, h1, h2, ldh, w,         \
                      partial, ldp, cnt, m, j, st, rtol, maxit);
    SD_AR_CASES(SD_AR_AN)
#undef SD_AR_AN
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t fg_update(int ninst, int m, int j, const FgState& st, const double* h1, const double* h2, int ldh,
                      double rtol, int maxit, cudaStream_t s) {
  // stat[j] collects the running flags of all instances
  cudaError_t e = cudaMemsetAsync(st.stat + j, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const size_t shm = sizeof(double) * (3 * (size_t)m + 2);
  SD_LAUNCH(k_fg_update, ninst, 64, shm, s, ninst, m, j, st, h1, h2, ldh, rtol, maxit);
  return cudaGetLastError();
}
cudaError_t fg_solve(int ninst, int m, const FgState& st, int ldh, cudaStream_t s) {
  SD_LAUNCH(k_fg_solve, (ninst + 127) / 128, 128, 0, s, ninst, m, st, ldh);
  return cudaGetLastError();
}
cudaError_t seg_mul(int nchunks, const int64_t* cbeg, const int64_t* cend, const int* cseg, const double* in,
                    double* out, const double* f, cudaStream_t s, float* out32) {
  if (nchunks == 0) return cudaSuccess;
  SD_LAUNCH(k_seg_mul, nchunks, 256, 0, s, cbeg, cend, cseg, in, out, f, out32);
  return cudaGetLastError();
}

}  // namespace sd
