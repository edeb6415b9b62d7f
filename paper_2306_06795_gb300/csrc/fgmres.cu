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
// One block per instance: the column and the previous rotations are staged
// in shared memory by all threads, thread 0 applies the rotations in order,
// and the running flags are OR-ed into stat[j] (zeroed beforehand).
__global__ void __launch_bounds__(64) k_fg_update(int ninst, int m, int j, FgState st, const double* __restrict__ h1buf,
                            const double* __restrict__ h2buf, int ldh, double rtol, int maxit) {
  extern __shared__ double fsm[];
  double* col = fsm;            // [j+2]
  double* csS = col + (m + 2);  // [j]
  double* snS = csS + m;        // [j]
  __shared__ double wmax[2];
  const int s = blockIdx.x;
  if (s >= ninst) return;
  if (!st.run[s]) {  // block-uniform
    if (threadIdx.x == 0) st.scale[s] = 0.0;
    return;
  }
  double* H = st.H + (size_t)s * (m + 1) * m;
  double* cs = st.cs + (size_t)s * m;
  double* sn = st.sn + (size_t)s * m;
  const double* h1 = h1buf + (size_t)s * ldh;
  const double* h2 = h2buf + (size_t)s * ldh;
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
    const double hmax = fmax(wmax[0], wmax[1]);
    double* g = st.g + (size_t)s * (m + 1);
    const double hn = sqrt(h1[j + 1]);
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
  // stat[j] collects the running flags of all instances
  cudaError_t e = cudaMemsetAsync(st.stat + j, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const size_t shm = sizeof(double) * (3 * (size_t)m + 2);
  k_fg_update<<<ninst, 64, shm, s>>>(ninst, m, j, st, h1, h2, ldh, rtol, maxit);
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
