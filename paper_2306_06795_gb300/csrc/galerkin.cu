// Device-side Galerkin product of the AMG setup (Alg. 1: the coarse
// operator K_{l+1} = P_l^T K_l P_l), FP64 and deterministic.
//
// P^T is formed by a counting transpose whose rows are then sorted by
// column.  Each sparse product A B (row-wise, Gustavson) runs one warp per
// output row: the row's partial products a_ik b_kj are listed in a fixed
// order (k ascending along A's row, then j along B's row k), sorted in
// shared memory by (j, list position) with a bitonic network, and equal
// columns are summed in list order.  A symbolic pass counts each row's
// distinct columns (row pointers by a prefix sum), a numeric pass writes
// them, sorted.  Results therefore do not depend on thread timing.
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

}  // namespace sd
