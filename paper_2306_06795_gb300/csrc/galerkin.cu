// Device-side steps of the AMG setup (Alg. 1), FP64 and deterministic: the
// Galerkin product K_{l+1} = P_l^T K_l P_l, the strength of connection,
// the tentative prolongator of given aggregates, the Jacobi-smoothed
// prolongator, and the Vanka patch lists of a Galerkin level (Sec. 3.3.1).
// The greedy aggregation and the spectral-radius estimate stay on the host.
//
// P^T is formed by a counting transpose whose rows are then sorted by
// column.  Each sparse product A B (row-wise, Gustavson) runs one warp per
// output row: the row's partial products a_ik b_kj are listed in a fixed
// order (k ascending along A's row, then j along B's row k), sorted in
// shared memory by (j, list position) with a bitonic network, and equal
// columns are summed in list order.  A symbolic pass counts each row's
// distinct columns (row pointers by a prefix sum), a numeric pass writes
// them, sorted.  Results therefore do not depend on thread timing.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "common.cuh"

namespace sd {

constexpr int kGalCap = 4096;  // partial products per output row (shared-memory sort capacity)

namespace {

__global__ void k_count_cols(int nrows, const int64_t* __restrict__ rp, const int* __restrict__ col,
                             int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) atomicAdd(cnt + col[k], 1);
}

__global__ void k_transpose_fill(int nrows, const int64_t* __restrict__ rp, const int* __restrict__ col,
                                 const double* __restrict__ val, int64_t* __restrict__ cursor,
                                 int* __restrict__ tcol, double* __restrict__ tval) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
    const int64_t pos = atomicAdd(reinterpret_cast<unsigned long long*>(cursor + col[k]), 1ull);
    tcol[pos] = i;
    tval[pos] = val[k];
  }
}

// rows of a transpose: insertion sort by column (rows are short), one thread per row
__global__ void k_sort_rows(int nrows, const int64_t* __restrict__ rp, int* __restrict__ col,
                            double* __restrict__ val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows) return;
  const int64_t b = rp[i], e = rp[i + 1];
  for (int64_t k = b + 1; k < e; ++k) {
    const int c = col[k];
    const double v = val[k];
    int64_t q = k - 1;
    while (q >= b && col[q] > c) {
      col[q + 1] = col[q];
      val[q + 1] = val[q];
      --q;
    }
    col[q + 1] = c;
    val[q + 1] = v;
  }
}

// One warp per output row of A B.  pass 0: count distinct columns into
// cnt[i]; pass 1: write them (sorted) at rp_c[i].  err: a row over kGalCap.
__global__ void __launch_bounds__(32) k_spgemm_row(int nrows, const int64_t* __restrict__ ra,
    const int* __restrict__ ca, const double* __restrict__ va, const int64_t* __restrict__ rb,
    const int* __restrict__ cb, const double* __restrict__ vb, int pass, int64_t* __restrict__ cnt,
    const int64_t* __restrict__ rc, int* __restrict__ cc, double* __restrict__ vc, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char gsm[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(gsm);       // (j << 32) | position
  double* pv = reinterpret_cast<double*>(key + kGalCap);                    // products by position
  const int i = blockIdx.x;
  const int lane = threadIdx.x;
  if (i >= nrows) return;
  const int64_t a0 = ra[i], a1 = ra[i + 1];
  // list the products in order: for each entry k of A's row, B's row k
  int base = 0;
  for (int64_t ka0 = a0; ka0 < a1; ka0 += 32) {
    const int64_t ka = ka0 + lane;
    const int k = ka < a1 ? ca[ka] : 0;
    const int len = ka < a1 ? (int)(rb[k + 1] - rb[k]) : 0;
    // inclusive scan of the lengths over the warp
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (base + total > kGalCap) {
      if (lane == 0) atomicOr(err, 1);
      return;
    }
    const int start = base + incl - len;
    if (ka < a1) {
      const double a = va[ka];
      for (int q = 0; q < len; ++q) {
        const int64_t kb = rb[k] + q;
        key[start + q] = ((unsigned long long)(unsigned)cb[kb] << 32) | (unsigned)(start + q);
        pv[start + q] = a * vb[kb];
      }
    }
    base += total;
  }
  const int np = base;
  int sz = 1;
  while (sz < np) sz <<= 1;
  for (int p = np + lane; p < sz; p += 32) key[p] = ~0ull;
  __syncwarp();
  // bitonic sort of key[0 .. sz)
  for (int k2 = 2; k2 <= sz; k2 <<= 1)
    for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
      for (int t = lane; t < sz; t += 32) {
        const int u = t ^ j2;
        if (u > t) {
          const unsigned long long x = key[t], y = key[u];
          const bool up = (t & k2) == 0;
          if ((x > y) == up) {
            key[t] = y;
            key[u] = x;
          }
        }
      }
      __syncwarp();
    }
  // distinct columns: position p starts a run when its column differs from p-1
  if (pass == 0) {
    int distinct = 0;
    for (int p = lane; p < np; p += 32)
      distinct += (p == 0 || (key[p] >> 32) != (key[p - 1] >> 32)) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) distinct += __shfl_xor_sync(0xffffffffu, distinct, o);
    if (lane == 0) cnt[i] = distinct;
    return;
  }
  // pass 1: lane 0 walks the sorted list, summing each run in list order
  if (lane == 0) {
    int64_t o = rc[i];
    int p = 0;
    while (p < np) {
      const unsigned j = (unsigned)(key[p] >> 32);
      double s = 0.0;
      while (p < np && (unsigned)(key[p] >> 32) == j) {
        s += pv[(unsigned)(key[p] & 0xffffffffu)];
        ++p;
      }
      cc[o] = (int)j;
      vc[o] = s;
      ++o;
    }
  }
}

struct DCSR {
  int n = 0, m = 0;
  int64_t nnz = 0;
  int64_t* rp = nullptr;
  int* col = nullptr;
  double* val = nullptr;
};

cudaError_t dcsr_alloc(DCSR& d, int n, int m, int64_t nnz) {
  d.n = n;
  d.m = m;
  d.nnz = nnz;
  cudaError_t e = cudaMalloc(&d.rp, sizeof(int64_t) * (n + 1));
  if (e == cudaSuccess) e = cudaMalloc(&d.col, sizeof(int) * (nnz > 0 ? nnz : 1));
  if (e == cudaSuccess) e = cudaMalloc(&d.val, sizeof(double) * (nnz > 0 ? nnz : 1));
  return e;
}
void dcsr_free(DCSR& d) {
  cudaFree(d.rp);
  cudaFree(d.col);
  cudaFree(d.val);
  d = DCSR();
}

// exclusive prefix sum on the host of n counts into rp (n+1), device copies
cudaError_t rows_from_counts(const int64_t* dcnt, int n, int64_t* drp, int64_t* nnz, cudaStream_t st) {
  std::vector<int64_t> c(n), r(n + 1, 0);
  cudaError_t e = cudaMemcpyAsync(c.data(), dcnt, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < n; ++i) r[i + 1] = r[i] + c[i];
  *nnz = r[n];
  e = cudaMemcpyAsync(drp, r.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t transpose(const DCSR& A, DCSR& T, cudaStream_t st) {
  int* cnt = nullptr;
  cudaError_t e = cudaMalloc(&cnt, sizeof(int) * (A.m > 0 ? A.m : 1));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(cnt, 0, sizeof(int) * (A.m > 0 ? A.m : 1), st);
  if (e == cudaSuccess && A.n > 0) {
    k_count_cols<<<(A.n + 255) / 256, 256, 0, st>>>(A.n, A.rp, A.col, cnt);
    e = cudaGetLastError();
  }
  std::vector<int> hc(A.m);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), cnt, sizeof(int) * A.m, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(cnt);
  if (e != cudaSuccess) return e;
  std::vector<int64_t> r(A.m + 1, 0);
  for (int j = 0; j < A.m; ++j) r[j + 1] = r[j] + hc[j];
  e = dcsr_alloc(T, A.m, A.n, r[A.m]);
  int64_t* cursor = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&cursor, sizeof(int64_t) * (A.m + 1));
  if (e == cudaSuccess) e = cudaMemcpyAsync(T.rp, r.data(), sizeof(int64_t) * (A.m + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cursor, r.data(), sizeof(int64_t) * (A.m + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && A.n > 0) {
    k_transpose_fill<<<(A.n + 255) / 256, 256, 0, st>>>(A.n, A.rp, A.col, A.val, cursor, T.col, T.val);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && T.n > 0) {
    k_sort_rows<<<(T.n + 255) / 256, 256, 0, st>>>(T.n, T.rp, T.col, T.val);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(cursor);
  return e;
}

// C = A B; status: 0, or 1 when a row has more than kGalCap partial products
cudaError_t spgemm(const DCSR& A, const DCSR& B, DCSR& C, int* status, cudaStream_t st) {
  *status = 0;
  int64_t* cnt = nullptr;
  int* err = nullptr;
  const size_t shm = (size_t)kGalCap * (sizeof(unsigned long long) + sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(k_spgemm_row, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(int64_t) * (A.n > 0 ? A.n : 1));
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess && A.n > 0) {
    k_spgemm_row<<<A.n, 32, shm, st>>>(A.n, A.rp, A.col, A.val, B.rp, B.col, B.val, 0, cnt, nullptr, nullptr,
                                        nullptr, err);
    e = cudaGetLastError();
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && herr) *status = 1;
  int64_t nnz = 0;
  if (e == cudaSuccess && !*status) {
    C.n = A.n;
    C.m = B.m;
    e = cudaMalloc(&C.rp, sizeof(int64_t) * (A.n + 1));
    if (e == cudaSuccess) e = rows_from_counts(cnt, A.n, C.rp, &nnz, st);
    C.nnz = nnz;
    if (e == cudaSuccess) e = cudaMalloc(&C.col, sizeof(int) * (nnz > 0 ? nnz : 1));
    if (e == cudaSuccess) e = cudaMalloc(&C.val, sizeof(double) * (nnz > 0 ? nnz : 1));
    if (e == cudaSuccess && A.n > 0) {
      k_spgemm_row<<<A.n, 32, shm, st>>>(A.n, A.rp, A.col, A.val, B.rp, B.col, B.val, 1, nullptr, C.rp, C.col,
                                          C.val, err);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(cnt);
  cudaFree(err);
  return e;
}

cudaError_t upload_dcsr(const int n, const int m, const int64_t* rp, const int* col, const double* val, DCSR& d,
                        cudaStream_t st) {
  const int64_t nnz = rp[n];
  cudaError_t e = dcsr_alloc(d, n, m, nnz);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d.rp, rp, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(d.col, col, sizeof(int) * nnz, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(d.val, val, sizeof(double) * nnz, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

}  // namespace

// Kc = P^T K P.  Host CSR in (validated by the caller), host arrays out
// (allocated here with new[]).  status: 0, or 1 for a row over the
// per-row product capacity.
cudaError_t galerkin_rap(int n, const int64_t* krp, const int* kcol, const double* kval, int nc, const int64_t* prp,
                         const int* pcol, const double* pval, cudaStream_t st, int* status, int64_t** crp,
                         int** ccol, double** cval, int64_t* cnnz) {
  DCSR K, P, Pt, T, C;
  *status = 0;
  cudaError_t e = upload_dcsr(n, n, krp, kcol, kval, K, st);
  if (e == cudaSuccess) e = upload_dcsr(n, nc, prp, pcol, pval, P, st);
  if (e == cudaSuccess) e = transpose(P, Pt, st);
  if (e == cudaSuccess) e = spgemm(K, P, T, status, st);
  if (e == cudaSuccess && !*status) e = spgemm(Pt, T, C, status, st);
  if (e == cudaSuccess && !*status) {
    *cnnz = C.nnz;
    *crp = new int64_t[(size_t)nc + 1];
    *ccol = new int[(size_t)(C.nnz > 0 ? C.nnz : 1)];
    *cval = new double[(size_t)(C.nnz > 0 ? C.nnz : 1)];
    e = cudaMemcpyAsync(*crp, C.rp, sizeof(int64_t) * (nc + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && C.nnz) e = cudaMemcpyAsync(*ccol, C.col, sizeof(int) * C.nnz, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && C.nnz)
      e = cudaMemcpyAsync(*cval, C.val, sizeof(double) * C.nnz, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  dcsr_free(K);
  dcsr_free(P);
  dcsr_free(Pt);
  dcsr_free(T);
  dcsr_free(C);
  return e;
}

// ------------------------------------------------------------ SA steps
namespace {

// |a_ii| per row (0 when no diagonal is stored) and whether the row stores a
// nonzero off-diagonal entry
__global__ void k_row_diag(int n, const int64_t* __restrict__ rp, const int* __restrict__ col,
                           const double* __restrict__ val, double* __restrict__ diag, int* __restrict__ offd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  int od = 0;
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
    if (col[k] == i) d = val[k];
    else if (val[k] != 0.0) od = 1;
  }
  diag[i] = d;
  offd[i] = od;
}

// Strength of connection: off-diagonal j is strong for row i when
// |a_ij| > theta sqrt(|a_ii| |a_jj|).  pass 0 counts, pass 1 writes (value 1).
__global__ void k_strength(int n, const int64_t* __restrict__ rp, const int* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ diag, double theta, int pass,
                           int64_t* __restrict__ cnt, const int64_t* __restrict__ srp, int* __restrict__ scol,
                           double* __restrict__ sval) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t c = 0, o = pass ? srp[i] : 0;
  const double di = fabs(diag[i]);
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
    const int j = col[k];
    if (j == i) continue;
    const double bound = __dmul_rn(theta, sqrt(__dmul_rn(di, fabs(diag[j]))));
    if (fabs(val[k]) > bound) {
      if (pass) {
        scol[o] = j;
        sval[o] = 1.0;
        ++o;
      } else {
        ++c;
      }
    }
  }
  if (!pass) cnt[i] = c;
}

__global__ void k_agg_count(int n, const int* __restrict__ agg, int* __restrict__ cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && agg[i] >= 0) atomicAdd(cnt + agg[i], 1);
}

__global__ void k_agg_fill(int n, const int* __restrict__ agg, int64_t* __restrict__ cursor,
                           int* __restrict__ members) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || agg[i] < 0) return;
  const int64_t pos = atomicAdd(reinterpret_cast<unsigned long long*>(cursor + agg[i]), 1ull);
  members[pos] = i;
}

// Per aggregate: members sorted ascending, then ||B restricted||_2 summed
// in node order (products and sums rounded separately, no fused multiply-add)
__global__ void k_agg_norm(int na, const int64_t* __restrict__ arp, int* __restrict__ members,
                           const double* __restrict__ B, double* __restrict__ nrm) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= na) return;
  const int64_t b = arp[a], e = arp[a + 1];
  for (int64_t k = b + 1; k < e; ++k) {
    const int v = members[k];
    int64_t q = k - 1;
    while (q >= b && members[q] > v) {
      members[q + 1] = members[q];
      --q;
    }
    members[q + 1] = v;
  }
  double s = 0.0;
  for (int64_t k = b; k < e; ++k) {
    const double x = B[members[k]];
    s = __dadd_rn(s, __dmul_rn(x, x));
  }
  nrm[a] = sqrt(s);
}

// T: row i has the one entry (agg_i, B_i / ||B|| of its aggregate); rows
// outside every aggregate are empty.  trp is the prefix count of aggregated rows.
__global__ void k_tentative(int n, const int* __restrict__ agg, const double* __restrict__ B,
                            const double* __restrict__ nrm, const int64_t* __restrict__ trp, int* __restrict__ tcol,
                            double* __restrict__ tval) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || agg[i] < 0) return;
  tcol[trp[i]] = agg[i];
  tval[trp[i]] = B[i] / nrm[agg[i]];
}

// P = T - omega D^-1 (A T) on the union of the two sorted row patterns,
// entries that come out exactly zero dropped; D^-1 is zero on rows with no
// nonzero off-diagonal entry.  Each entry: t - omega (dinv_i (A T)_ij).
__global__ void k_smooth_merge(int n, const int64_t* __restrict__ trp, const int* __restrict__ tcol,
                               const double* __restrict__ tval, const int64_t* __restrict__ arp,
                               const int* __restrict__ acol, const double* __restrict__ aval,
                               const double* __restrict__ diag, const int* __restrict__ offd, double omega, int pass,
                               int64_t* __restrict__ cnt, const int64_t* __restrict__ prp, int* __restrict__ pcol,
                               double* __restrict__ pval) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double dinv = offd[i] ? 1.0 / diag[i] : 0.0;
  int64_t p = trp[i], q = arp[i], o = pass ? prp[i] : 0, c = 0;
  const int64_t pe = trp[i + 1], qe = arp[i + 1];
  while (p < pe || q < qe) {
    const int jt = p < pe ? tcol[p] : 0x7fffffff, ja = q < qe ? acol[q] : 0x7fffffff;
    const int j = jt < ja ? jt : ja;
    const double t = jt == j ? tval[p] : 0.0;
    const double y = ja == j ? __dmul_rn(omega, __dmul_rn(dinv, aval[q])) : 0.0;
    const double v = __dsub_rn(t, y);
    if (jt == j) ++p;
    if (ja == j) ++q;
    if (v == 0.0) continue;
    if (pass) {
      pcol[o] = j;
      pval[o] = v;
      ++o;
    } else {
      ++c;
    }
  }
  if (!pass) cnt[i] = c;
}

constexpr int kPatchCap = 4096;  // velocity entries of one pressure row

// Vanka patch of pressure row s (one warp): the velocity nodes whose largest
// |b| over the components exceeds rel_tol times the row's largest, sorted.
// pass 0 counts the nodes, pass 1 writes them.  err: a row over kPatchCap.
__global__ void __launch_bounds__(32) k_patch_nodes(int npres, const int64_t* __restrict__ rp,
    const int* __restrict__ col, const double* __restrict__ val, const int64_t* __restrict__ off, int dim,
    double rel_tol, int pass, int64_t* __restrict__ cnt, const int64_t* __restrict__ nrp, int* __restrict__ nodes,
    int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char psm[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(psm);  // (node << 32) | position
  double* mag = reinterpret_cast<double*>(key + kPatchCap);
  const int s = blockIdx.x, lane = threadIdx.x;
  if (s >= npres) return;
  const int64_t row = off[dim] + s;
  const int64_t b = rp[row], e = rp[row + 1];
  const int64_t vel_end = off[dim];
  // velocity entries come first in the row (columns ascending): the first
  // pressure column by binary search
  int64_t lo = b, hi = e;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (col[mid] < vel_end) lo = mid + 1;
    else hi = mid;
  }
  const int nv = (int)(lo - b);
  if (nv > kPatchCap) {
    if (lane == 0) atomicOr(err, 1);
    return;
  }
  for (int k = lane; k < nv; k += 32) {
    const int cc = col[b + k];
    int c = 0;
    while (c + 1 < dim && cc >= off[c + 1]) ++c;
    key[k] = ((unsigned long long)(unsigned)(cc - (int)off[c]) << 32) | (unsigned)k;
    mag[k] = fabs(val[b + k]);
  }
  int sz = 1;
  while (sz < nv) sz <<= 1;
  for (int p = nv + lane; p < sz; p += 32) key[p] = ~0ull;
  __syncwarp();
  for (int k2 = 2; k2 <= sz; k2 <<= 1)
    for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
      for (int t = lane; t < sz; t += 32) {
        const int u = t ^ j2;
        if (u > t) {
          const unsigned long long x = key[t], y = key[u];
          const bool up = (t & k2) == 0;
          if ((x > y) == up) {
            key[t] = y;
            key[u] = x;
          }
        }
      }
      __syncwarp();
    }
  if (lane == 0) {
    double rowmax = 0.0;
    for (int k = 0; k < nv; ++k) rowmax = fmax(rowmax, mag[k]);
    const double thr = __dmul_rn(rel_tol, rowmax);
    int64_t o = pass ? nrp[s] : 0;
    int64_t c = 0;
    int p = 0;
    while (p < nv) {
      const unsigned node = (unsigned)(key[p] >> 32);
      double m = 0.0;
      while (p < nv && (unsigned)(key[p] >> 32) == node) {
        m = fmax(m, mag[(unsigned)(key[p] & 0xffffffffu)]);
        ++p;
      }
      if (m > thr) {
        if (pass) nodes[o++] = (int)node;
        else ++c;
      }
    }
    if (!pass) cnt[s] = c;
  }
}

__global__ void k_patch_lists(int npres, int dim, const int64_t* __restrict__ off, const int64_t* __restrict__ nrp,
                              const int* __restrict__ nodes, int64_t* __restrict__ ptr, int* __restrict__ dof,
                              int* __restrict__ nvel, int* __restrict__ npr) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= npres) return;
  const int64_t n0 = nrp[s], m = nrp[s + 1] - nrp[s];
  const int64_t o = ptr[s];
  for (int c = 0; c < dim; ++c) {
    for (int64_t k = 0; k < m; ++k) dof[o + c * m + k] = (int)(off[c] + nodes[n0 + k]);
    nvel[(int64_t)s * dim + c] = (int)m;
  }
  dof[o + dim * m] = (int)(off[dim] + s);
  npr[s] = 1;
}

cudaError_t download_dcsr(const DCSR& C, int64_t** crp, int** ccol, double** cval, cudaStream_t st) {
  *crp = new int64_t[(size_t)C.n + 1];
  *ccol = new int[(size_t)(C.nnz > 0 ? C.nnz : 1)];
  *cval = new double[(size_t)(C.nnz > 0 ? C.nnz : 1)];
  cudaError_t e = cudaMemcpyAsync(*crp, C.rp, sizeof(int64_t) * (C.n + 1), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && C.nnz) e = cudaMemcpyAsync(*ccol, C.col, sizeof(int) * C.nnz, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && C.nnz) e = cudaMemcpyAsync(*cval, C.val, sizeof(double) * C.nnz, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

// counts -> row pointers (device), then allocate columns and values
cudaError_t alloc_from_counts(DCSR& C, int n, int m, const int64_t* dcnt, cudaStream_t st) {
  C.n = n;
  C.m = m;
  int64_t nnz = 0;
  cudaError_t e = cudaMalloc(&C.rp, sizeof(int64_t) * (n + 1));
  if (e == cudaSuccess) e = rows_from_counts(dcnt, n, C.rp, &nnz, st);
  C.nnz = nnz;
  if (e == cudaSuccess) e = cudaMalloc(&C.col, sizeof(int) * (nnz > 0 ? nnz : 1));
  if (e == cudaSuccess) e = cudaMalloc(&C.val, sizeof(double) * (nnz > 0 ? nnz : 1));
  return e;
}

inline unsigned nblk(int n) { return (unsigned)((n + 255) / 256); }

}  // namespace

// Strength of connection of A (n x n host CSR): pattern S, values 1.
cudaError_t sa_strength(int n, const int64_t* rp, const int* col, const double* val, double theta, cudaStream_t st,
                        int64_t** srp, int** scol, double** sval, int64_t* snnz) {
  DCSR A, S;
  double* diag = nullptr;
  int* offd = nullptr;
  int64_t* cnt = nullptr;
  cudaError_t e = upload_dcsr(n, n, rp, col, val, A, st);
  if (e == cudaSuccess) e = cudaMalloc(&diag, sizeof(double) * (n > 0 ? n : 1));
  if (e == cudaSuccess) e = cudaMalloc(&offd, sizeof(int) * (n > 0 ? n : 1));
  if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(int64_t) * (n > 0 ? n : 1));
  if (e == cudaSuccess && n > 0) {
    k_row_diag<<<nblk(n), 256, 0, st>>>(n, A.rp, A.col, A.val, diag, offd);
    k_strength<<<nblk(n), 256, 0, st>>>(n, A.rp, A.col, A.val, diag, theta, 0, cnt, nullptr, nullptr, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = alloc_from_counts(S, n, n, cnt, st);
  if (e == cudaSuccess && n > 0) {
    k_strength<<<nblk(n), 256, 0, st>>>(n, A.rp, A.col, A.val, diag, theta, 1, nullptr, S.rp, S.col, S.val);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    *snnz = S.nnz;
    e = download_dcsr(S, srp, scol, sval, st);
  }
  cudaFree(diag);
  cudaFree(offd);
  cudaFree(cnt);
  dcsr_free(A);
  dcsr_free(S);
  return e;
}

// Tentative prolongator of aggregates agg (n, -1 outside every aggregate)
// with near-null vector B: T (n x na) and the aggregate norms Bc (host, na).
cudaError_t sa_tentative(int n, const int* agg, int na, const double* B, cudaStream_t st, int64_t** trp, int** tcol,
                         double** tval, int64_t* tnnz, double* Bc) {
  int *dagg = nullptr, *acnt = nullptr, *members = nullptr;
  double *dB = nullptr, *nrm = nullptr;
  int64_t *arp = nullptr, *cursor = nullptr;
  DCSR T;
  std::vector<int> hcnt(na > 0 ? na : 1);
  std::vector<int64_t> ar((size_t)na + 1, 0), tr((size_t)n + 1, 0);
  for (int i = 0; i < n; ++i) tr[i + 1] = tr[i] + (agg[i] >= 0 ? 1 : 0);
  cudaError_t e = cudaMalloc(&dagg, sizeof(int) * (n > 0 ? n : 1));
  if (e == cudaSuccess) e = cudaMalloc(&dB, sizeof(double) * (n > 0 ? n : 1));
  if (e == cudaSuccess) e = cudaMalloc(&acnt, sizeof(int) * (na > 0 ? na : 1));
  if (e == cudaSuccess) e = cudaMalloc(&nrm, sizeof(double) * (na > 0 ? na : 1));
  if (e == cudaSuccess) e = cudaMalloc(&arp, sizeof(int64_t) * (na + 1));
  if (e == cudaSuccess) e = cudaMalloc(&cursor, sizeof(int64_t) * (na + 1));
  if (e == cudaSuccess) e = cudaMalloc(&members, sizeof(int) * (tr[n] > 0 ? tr[n] : 1));
  if (e == cudaSuccess && n) e = cudaMemcpyAsync(dagg, agg, sizeof(int) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n) e = cudaMemcpyAsync(dB, B, sizeof(double) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(acnt, 0, sizeof(int) * (na > 0 ? na : 1), st);
  if (e == cudaSuccess && n > 0) {
    k_agg_count<<<nblk(n), 256, 0, st>>>(n, dagg, acnt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && na) e = cudaMemcpyAsync(hcnt.data(), acnt, sizeof(int) * na, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  for (int a = 0; a < na; ++a) ar[a + 1] = ar[a] + hcnt[a];
  if (e == cudaSuccess) e = cudaMemcpyAsync(arp, ar.data(), sizeof(int64_t) * (na + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cursor, ar.data(), sizeof(int64_t) * (na + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n > 0) {
    k_agg_fill<<<nblk(n), 256, 0, st>>>(n, dagg, cursor, members);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && na > 0) {
    k_agg_norm<<<nblk(na), 256, 0, st>>>(na, arp, members, dB, nrm);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = dcsr_alloc(T, n, na, tr[n]);
  if (e == cudaSuccess) e = cudaMemcpyAsync(T.rp, tr.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && n > 0) {
    k_tentative<<<nblk(n), 256, 0, st>>>(n, dagg, dB, nrm, T.rp, T.col, T.val);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && na) e = cudaMemcpyAsync(Bc, nrm, sizeof(double) * na, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) {
    *tnnz = T.nnz;
    e = download_dcsr(T, trp, tcol, tval, st);
  }
  cudaFree(dagg);
  cudaFree(dB);
  cudaFree(acnt);
  cudaFree(nrm);
  cudaFree(arp);
  cudaFree(cursor);
  cudaFree(members);
  dcsr_free(T);
  return e;
}

// Jacobi-smoothed prolongator P = T - omega D^-1 A T (A n x n, T n x nc).
cudaError_t sa_smooth(int n, const int64_t* arp, const int* acol, const double* aval, int nc, const int64_t* trp,
                      const int* tcol, const double* tval, double omega, cudaStream_t st, int* status,
                      int64_t** prp, int** pcol, double** pval, int64_t* pnnz) {
  DCSR A, T, AT, P;
  double* diag = nullptr;
  int* offd = nullptr;
  int64_t* cnt = nullptr;
  *status = 0;
  cudaError_t e = upload_dcsr(n, n, arp, acol, aval, A, st);
  if (e == cudaSuccess) e = upload_dcsr(n, nc, trp, tcol, tval, T, st);
  if (e == cudaSuccess) e = spgemm(A, T, AT, status, st);
  if (e == cudaSuccess && !*status) {
    e = cudaMalloc(&diag, sizeof(double) * (n > 0 ? n : 1));
    if (e == cudaSuccess) e = cudaMalloc(&offd, sizeof(int) * (n > 0 ? n : 1));
    if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(int64_t) * (n > 0 ? n : 1));
    if (e == cudaSuccess && n > 0) {
      k_row_diag<<<nblk(n), 256, 0, st>>>(n, A.rp, A.col, A.val, diag, offd);
      k_smooth_merge<<<nblk(n), 256, 0, st>>>(n, T.rp, T.col, T.val, AT.rp, AT.col, AT.val, diag, offd, omega, 0,
                                              cnt, nullptr, nullptr, nullptr);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = alloc_from_counts(P, n, nc, cnt, st);
    if (e == cudaSuccess && n > 0) {
      k_smooth_merge<<<nblk(n), 256, 0, st>>>(n, T.rp, T.col, T.val, AT.rp, AT.col, AT.val, diag, offd, omega, 1,
                                              nullptr, P.rp, P.col, P.val);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      *pnnz = P.nnz;
      e = download_dcsr(P, prp, pcol, pval, st);
    }
  }
  cudaFree(diag);
  cudaFree(offd);
  cudaFree(cnt);
  dcsr_free(A);
  dcsr_free(T);
  dcsr_free(AT);
  dcsr_free(P);
  return e;
}

// Vanka patch lists of a Galerkin level: one patch per pressure DoF s (seed
// off[dim] + s) holding every velocity node linked to it by an entry of B
// above rel_tol times the row's largest, with all dim components.
// status: 1 when a pressure row has more than kPatchCap velocity entries.
cudaError_t vanka_patch_lists(int n, const int64_t* rp, const int* col, const double* val, const int64_t* hoff, int dim,
                              double rel_tol, cudaStream_t st, int* status, int* npatch, int64_t** hptr, int** hdof,
                              int** hnvel, int** hnpres) {
  DCSR K;
  int64_t *off = nullptr, *cnt = nullptr, *nrp = nullptr, *ptr = nullptr;
  int *nodes = nullptr, *dof = nullptr, *nvel = nullptr, *npr = nullptr, *err = nullptr;
  *status = 0;
  const int np = (int)(hoff[dim + 1] - hoff[dim]);
  *npatch = np;
  const size_t shm = (size_t)kPatchCap * (sizeof(unsigned long long) + sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(k_patch_nodes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (e == cudaSuccess) e = upload_dcsr(n, n, rp, col, val, K, st);
  if (e == cudaSuccess) e = cudaMalloc(&off, sizeof(int64_t) * (dim + 2));
  if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(int64_t) * (np > 0 ? np : 1));
  if (e == cudaSuccess) e = cudaMalloc(&nrp, sizeof(int64_t) * (np + 1));
  if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(off, hoff, sizeof(int64_t) * (dim + 2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && np > 0) {
    k_patch_nodes<<<np, 32, shm, st>>>(np, K.rp, K.col, K.val, off, dim, rel_tol, 0, cnt, nullptr, nullptr, err);
    e = cudaGetLastError();
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && herr) *status = 1;
  int64_t nn = 0;
  if (e == cudaSuccess && !*status) e = rows_from_counts(cnt, np, nrp, &nn, st);
  std::vector<int64_t> hn((size_t)np + 1), hp((size_t)np + 1, 0);
  if (e == cudaSuccess && !*status) {
    e = cudaMemcpyAsync(hn.data(), nrp, sizeof(int64_t) * (np + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int s2 = 0; s2 < np; ++s2) hp[s2 + 1] = hp[s2] + dim * (hn[s2 + 1] - hn[s2]) + 1;
    if (e == cudaSuccess) e = cudaMalloc(&nodes, sizeof(int) * (nn > 0 ? nn : 1));
    if (e == cudaSuccess) e = cudaMalloc(&ptr, sizeof(int64_t) * (np + 1));
    if (e == cudaSuccess) e = cudaMalloc(&dof, sizeof(int) * (hp[np] > 0 ? hp[np] : 1));
    if (e == cudaSuccess) e = cudaMalloc(&nvel, sizeof(int) * ((size_t)np * dim > 0 ? (size_t)np * dim : 1));
    if (e == cudaSuccess) e = cudaMalloc(&npr, sizeof(int) * (np > 0 ? np : 1));
    if (e == cudaSuccess) e = cudaMemcpyAsync(ptr, hp.data(), sizeof(int64_t) * (np + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && np > 0) {
      k_patch_nodes<<<np, 32, shm, st>>>(np, K.rp, K.col, K.val, off, dim, rel_tol, 1, nullptr, nrp, nodes, err);
      k_patch_lists<<<nblk(np), 256, 0, st>>>(np, dim, off, nrp, nodes, ptr, dof, nvel, npr);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      *hptr = new int64_t[(size_t)np + 1];
      *hdof = new int[(size_t)(hp[np] > 0 ? hp[np] : 1)];
      *hnvel = new int[(size_t)np * dim + 1];
      *hnpres = new int[(size_t)np + 1];
      std::copy(hp.begin(), hp.end(), *hptr);
      if (hp[np]) e = cudaMemcpyAsync(*hdof, dof, sizeof(int) * hp[np], cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess && np)
        e = cudaMemcpyAsync(*hnvel, nvel, sizeof(int) * (size_t)np * dim, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess && np) e = cudaMemcpyAsync(*hnpres, npr, sizeof(int) * np, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
  }
  cudaFree(off);
  cudaFree(cnt);
  cudaFree(nrp);
  cudaFree(ptr);
  cudaFree(nodes);
  cudaFree(dof);
  cudaFree(nvel);
  cudaFree(npr);
  cudaFree(err);
  dcsr_free(K);
  return e;
}

}  // namespace sd
