// Device-side bookkeeping of restarted FGMRES (Sec. 4): per instance, the
// Hessenberg column, Givens rotations, the residual estimate, the running
// flag and the scale of the next Krylov vector are updated by one thread,
// so an Arnoldi step needs no host round trip.  One block handles every
// instance; its flag reduction and all arithmetic run in a fixed order.
#include <cmath>

#include "common.cuh"

namespace sd {


// Start of a restart cycle: h[s*ldh] = ||r_s||^2.
__global__ void __launch_bounds__(256) k_fg_start(int ninst, int m, FgState st, const double* __restrict__ h, int ldh, double rtol, int maxit,
                           int first) {
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

// Arnoldi step j: column j of H from the two Gram-Schmidt passes (h1 in
// h1buf, h2 in h2buf, ||w||^2 in h1buf[j+1]), Givens update, convergence.
__global__ void __launch_bounds__(256) k_fg_update(int ninst, int m, int j, FgState st, const double* __restrict__ h1buf,
                            const double* __restrict__ h2buf, int ldh, double rtol, int maxit) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < ninst; s += blockDim.x) {
    if (!st.run[s]) {
      st.scale[s] = 0.0;
      continue;
    }
    double* H = st.H + (size_t)s * (m + 1) * m;
    double* cs = st.cs + (size_t)s * m;
    double* sn = st.sn + (size_t)s * m;
    double* g = st.g + (size_t)s * (m + 1);
    const double* h1 = h1buf + (size_t)s * ldh;
    const double* h2 = h2buf + (size_t)s * ldh;
    double hmax = 0.0;
    for (int i = 0; i <= j; ++i) {
      H[i * m + j] = h1[i] + h2[i];
      hmax = fmax(hmax, fabs(H[i * m + j]));
    }
    const double hn = sqrt(h1[j + 1]);
    H[(j + 1) * m + j] = hn;
    const bool breakdown = !(hn > 1e-14 * fmax(hmax, 1e-300));
    for (int i = 0; i < j; ++i) {
      const double t = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
      H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
      H[i * m + j] = t;
    }
    const double den = hypot(H[j * m + j], H[(j + 1) * m + j]);
    cs[j] = H[j * m + j] / den;
    sn[j] = H[(j + 1) * m + j] / den;
    H[j * m + j] = den;
    H[(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    st.its[s] += 1;
    st.kcol[s] = j + 1;
    if (!isfinite(g[j + 1])) atomicOr(st.err, 1);
    const bool run = !(fabs(g[j + 1]) <= rtol * st.bnorm[s]) && !breakdown && st.its[s] < maxit && j + 1 < m &&
                     isfinite(g[j + 1]);
    st.run[s] = run;
    st.scale[s] = run ? 1.0 / hn : 0.0;
    if (run) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) st.stat[j] = any;
}

// y of the least-squares problem by back substitution (per instance).
__global__ void k_fg_solve(int ninst, int m, FgState st, int ldh) {
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

// out[row] = in[row] * f[seg(row)]
__global__ void __launch_bounds__(256) k_seg_mul(const int64_t* __restrict__ cbeg, const int64_t* __restrict__ cend,
                                                 const int* __restrict__ cseg, const double* __restrict__ in,
                                                 double* __restrict__ out, const double* __restrict__ f) {
  const int c = blockIdx.x;
  const double v = f[cseg[c]];
  for (int64_t r = cbeg[c] + threadIdx.x; r < cend[c]; r += 256) out[r] = v == 0.0 ? 0.0 : in[r] * v;
}

cudaError_t fg_start(int ninst, int m, const FgState& st, const double* h, int ldh, double rtol, int maxit, int first,
                     cudaStream_t s) {
  k_fg_start<<<1, 256, 0, s>>>(ninst, m, st, h, ldh, rtol, maxit, first);
  return cudaGetLastError();
}
cudaError_t fg_update(int ninst, int m, int j, const FgState& st, const double* h1, const double* h2, int ldh,
                      double rtol, int maxit, cudaStream_t s) {
  k_fg_update<<<1, 256, 0, s>>>(ninst, m, j, st, h1, h2, ldh, rtol, maxit);
  return cudaGetLastError();
}
cudaError_t fg_solve(int ninst, int m, const FgState& st, int ldh, cudaStream_t s) {
  k_fg_solve<<<(ninst + 127) / 128, 128, 0, s>>>(ninst, m, st, ldh);
  return cudaGetLastError();
}
cudaError_t seg_mul(int nchunks, const int64_t* cbeg, const int64_t* cend, const int* cseg, const double* in,
                    double* out, const double* f, cudaStream_t s) {
  if (nchunks == 0) return cudaSuccess;
  k_seg_mul<<<nchunks, 256, 0, s>>>(cbeg, cend, cseg, in, out, f);
  return cudaGetLastError();
}

}  // namespace sd
