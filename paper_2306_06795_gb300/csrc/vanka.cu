// Additive Vanka relaxation on the device (Sec. 3.3.1): batched patch
// factorisation (step a5), gather + block-factorised patch solve (a4, a6)
// and the deterministic weighted scatter (a7).
//
// Patch factor layout (elements of T, block start 16-byte aligned):
//   nblk blocks A_c^-1 (nblk = 1 when all velocity components share one
//   block, else dim): for the patches of the bulk-copy bins a packed lower
//   triangle, m(m+1)/2 entries row by row; for the rest the tiled lower
//   triangle of tiles.cuh; then U = A^-1 B^T stored seed-major (np columns
//   of dim*m); then S^-1 (np x np, row-major) with S = -B A^-1 B^T.
// The patch solve computes, for b = V_i r (Eqs. vanka_fact1/2),
//   y_u = A^-1 b_u,  y_p = S^-1 (b_p - U^T b_u),  x_u = y_u - U y_p,
// which is [I U^; 0 I][A^-1 0; B^ S^-1] b with U^ = -U and
// B^ = -S^-1 B A^-1 = -S^-1 U^T (A is symmetric), so B^ needs no storage.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "tiles.cuh"
#include "tma.cuh"

namespace sd {

constexpr int kWarpM = 32;    // velocity DoFs per component handled by the warp kernel
constexpr int kWarpPk = kWarpM * (kWarpM + 1) / 2;

__device__ __forceinline__ int packed_index(int a, int b) {
  return a >= b ? a * (a + 1) / 2 + b : b * (b + 1) / 2 + a;
}

// -------------------------------------------------------------- factorise
constexpr int kFacThreads = 256;  // CTA-per-patch factorisation (m > 32)

template <typename T>
__global__ void __launch_bounds__(kFacThreads) k_vanka_factor(int nlist, const int* __restrict__ list, int dim, int shared,
    const int* __restrict__ ptr, const int* __restrict__ dof, const int* __restrict__ nvel,
    const int* __restrict__ npres, const int64_t* __restrict__ foff, const int* __restrict__ rowptr,
    const int* __restrict__ col, const double* __restrict__ Kval, T* __restrict__ fac, int* nsing,
    int max_m, int max_np, T* __restrict__ gA, int nsmall) {
  pdl_enter();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if ((int)blockIdx.x >= nlist) return;
  const int i = list[blockIdx.x];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int base = ptr[i], m = nvel[i], np = npres[i];
  const int mu = dim * m, mt = mu + np;
  // shared layout (the m x m block lives in global scratch when gA is given)
  T* A = gA ? gA + (size_t)blockIdx.x * max_m * max_m : reinterpret_cast<T*>(smem_raw);
  T* BT = reinterpret_cast<T*>(smem_raw) + (gA ? 0 : (size_t)max_m * max_m);
  T* U = BT + (size_t)dim * max_m * max_np;
  T* colk = U + (size_t)dim * max_m * max_np;
  T* rowk = colk + max_m;
  T* S = rowk + max_m;               // kMaxNp^2
  T* misc = S + kMaxNp * kMaxNp;     // [0]: diag max, [1]: singular flag
  int* sdof = reinterpret_cast<int*>(misc + 4);

  for (int k = tid; k < mt; k += nt) sdof[k] = dof[base + k];
  for (int k = tid; k < mu * np; k += nt) BT[k] = T(0);
  if (tid == 0) misc[1] = T(0);
  __syncthreads();
  // B^T columns: entries of velocity rows in the seed (pressure) columns,
  // read eight at a time with all loads in flight
  for (int r = tid; r < mu; r += nt) {
    const int g = sdof[r];
    const int e1 = rowptr[g + 1];
    for (int e0 = rowptr[g]; e0 < e1; e0 += 8) {
      int cc[8];
      double vv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        cc[u] = e0 + u < e1 ? col[e0 + u] : -1;
        vv[u] = e0 + u < e1 ? Kval[e0 + u] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        for (int k = 0; k < np; ++k)
          if (sdof[mu + k] == cc[u]) BT[r * np + k] = T(vv[u]);
    }
  }
  const int nblk = shared ? 1 : dim;
  const bool tiled = i >= nsmall;
  const int64_t blk = tiled ? tiled_block_elems(m) : (int64_t)padded_pk<T>(m);
  T* out = fac + foff[i];
  for (int cb = 0; cb < nblk; ++cb) {
    __syncthreads();
    for (int e = tid; e < m * m; e += nt) A[e] = T(0);
    __syncthreads();
    for (int a = tid; a < m; a += nt) {
      const int g = sdof[cb * m + a];
      const int e1 = rowptr[g + 1];
      for (int e0 = rowptr[g]; e0 < e1; e0 += 8) {
        int cc[8];
        double vv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          cc[u] = e0 + u < e1 ? col[e0 + u] : -1;
          vv[u] = e0 + u < e1 ? Kval[e0 + u] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int pos = cc[u] >= 0 ? bsearch_int(sdof + cb * m, m, cc[u]) : -1;
          if (pos >= 0) A[a * m + pos] = T(vv[u]);
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      T dm = T(0);
      for (int a = 0; a < m; ++a) dm = fmax(dm, fabs(A[a * m + a]));
      misc[0] = dm;
    }
    __syncthreads();
    // Gauss-Jordan inversion in place; the block is SPD so no pivoting
    for (int k = 0; k < m; ++k) {
      T piv = A[k * m + k];
      const bool bad = !(fabs(piv) > T(1e-12) * misc[0]);
      if (bad) piv = T(1);  // keeps the arithmetic finite; the patch is flagged
      const T p = T(1) / piv;
      for (int j = tid; j < m; j += nt) {
        colk[j] = A[j * m + k];
        rowk[j] = (j == k) ? p : A[k * m + j] * p;
      }
      if (tid == 0 && bad) misc[1] = T(1);
      __syncthreads();
      // one warp per row, lanes along the row: no index division, conflict-free
      for (int ii = tid >> 5; ii < m; ii += nt >> 5) {
        const T ci = colk[ii];
        T* Ar = A + (size_t)ii * m;
        for (int jj = tid & 31; jj < m; jj += 32) {
          if (ii == k) Ar[jj] = rowk[jj];
          else if (jj == k) Ar[jj] = -ci * p;
          else Ar[jj] -= ci * rowk[jj];
        }
      }
      __syncthreads();
    }
    // lower triangle of the (symmetrised) inverse, tiled or packed
    if (tiled) {
      for (int64_t e = tid; e < blk; e += nt) {
        const int q = (int)(e >> 10);
        int I = 0;
        while ((I + 1) * (I + 2) / 2 <= q) ++I;
        const int J = q - I * (I + 1) / 2, r = (int)(e >> 5) & 31, c = ((int)e & 31) ^ r;
        const int a = I * 32 + r, b = J * 32 + c;
        out[cb * blk + e] = (a < m && b < m) ? T(0.5) * (A[a * m + b] + A[b * m + a]) : T(0);
      }
    } else {
      for (int a = tid; a < m; a += nt)
        for (int b = 0; b <= a; ++b) out[cb * blk + a * (a + 1) / 2 + b] = T(0.5) * (A[a * m + b] + A[b * m + a]);
    }
    // U rows of the components this block serves
    const int c0 = shared ? 0 : cb, c1 = shared ? dim : cb + 1;
    for (int c = c0; c < c1; ++c)
      for (int idx = tid; idx < m * np; idx += nt) {
        const int a = idx / np, k = idx - a * np;
        T s = T(0);
        for (int b = 0; b < m; ++b) s += A[a * m + b] * BT[(c * m + b) * np + k];
        U[(c * m + a) * np + k] = s;
      }
  }
  __syncthreads();
  if (tid < np * np) {
    const int k = tid / np, k2 = tid - k * np;
    T s = T(0);
    for (int r = 0; r < mu; ++r) s += BT[r * np + k] * U[r * np + k2];
    S[k * kMaxNp + k2] = -s;
  }
  __syncthreads();
  T* Uout = out + nblk * blk;
  T* Sout = Uout + mu * np;
  for (int idx = tid; idx < mu * np; idx += nt) {
    const int r = idx / np, k = idx - r * np;
    Uout[k * mu + r] = U[r * np + k];
  }
  if (tid == 0) {
    // S^-1 by Gauss-Jordan with partial pivoting (np <= 4)
    T M[kMaxNp][2 * kMaxNp];
    T smax = T(0);
    for (int a = 0; a < np; ++a)
      for (int b = 0; b < np; ++b) {
        M[a][b] = S[a * kMaxNp + b];
        M[a][np + b] = a == b ? T(1) : T(0);
        smax = fmax(smax, fabs(M[a][b]));
      }
    bool sing = misc[1] != T(0);
    for (int k = 0; k < np; ++k) {
      int pr = k;
      for (int a = k + 1; a < np; ++a)
        if (fabs(M[a][k]) > fabs(M[pr][k])) pr = a;
      if (!(fabs(M[pr][k]) > T(1e-12) * smax)) { sing = true; break; }
      if (pr != k)
        for (int b = 0; b < 2 * np; ++b) { T t = M[k][b]; M[k][b] = M[pr][b]; M[pr][b] = t; }
      const T p = T(1) / M[k][k];
      for (int b = 0; b < 2 * np; ++b) M[k][b] *= p;
      for (int a = 0; a < np; ++a)
        if (a != k) {
          const T f = M[a][k];
          for (int b = 0; b < 2 * np; ++b) M[a][b] -= f * M[k][b];
        }
    }
    for (int a = 0; a < np; ++a)
      for (int b = 0; b < np; ++b) Sout[a * np + b] = sing ? T(0) : M[a][np + b];
    if (sing) atomicAdd(nsing, 1);
  }
}

// One warp per patch for patches with m <= MAXM (8, 20 or 32) velocity DoFs
// per component: the same factorisation as above without block-wide
// barriers.  Lane a owns row a of the block in registers through the
// Gauss-Jordan sweep; at step k the pivot row goes to shared memory and
// every lane updates its row with one FMA per entry (the pivot lane's own
// scaling is written as the same update, row -= (1 - 1/p) row).
constexpr int kFacWarps = 4;

template <typename T, int MAXM>
struct FacWarpSmem {
  static constexpr int kDof = 3 * MAXM + kMaxNp;
  static constexpr int kStride = MAXM + 1;  // padded rows: conflict-free column reads
  __host__ __device__ static constexpr size_t bytes() {
    return ((size_t)kDof * sizeof(int) + 15) / 16 * 16 +
           sizeof(T) * ((size_t)MAXM * kStride + 2 * (size_t)3 * MAXM * kMaxNp + MAXM + kMaxNp * kMaxNp);
  }
};

template <typename T, int MAXM>
__global__ void __launch_bounds__(kFacWarps * 32) k_vanka_factor_warp(int nlist, const int* __restrict__ list,
    int dim, int shared, const int* __restrict__ ptr, const int* __restrict__ dof, const int* __restrict__ nvel,
    const int* __restrict__ npres, const int64_t* __restrict__ foff, const int* __restrict__ rowptr,
    const int* __restrict__ col, const double* __restrict__ Kval, T* __restrict__ fac, int* nsing, int nsmall) {
  pdl_enter();
  using L = FacWarpSmem<T, MAXM>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kFacWarps + warp;
  if (gw >= nlist) return;  // warp-uniform; no block barriers below
  unsigned char* mine = smem_raw + (size_t)warp * L::bytes();
  int* sdof = reinterpret_cast<int*>(mine);
  T* Am = reinterpret_cast<T*>(mine + ((size_t)L::kDof * sizeof(int) + 15) / 16 * 16);
  T* BT = Am + MAXM * L::kStride;
  T* U = BT + 3 * MAXM * kMaxNp;
  T* prow = U + 3 * MAXM * kMaxNp;
  T* S = prow + MAXM;
  const int i = list[gw];
  const int base = ptr[i], m = nvel[i], np = npres[i];
  const int mu = dim * m, mt = mu + np;
  for (int k = lane; k < mt; k += 32) sdof[k] = dof[base + k];
  for (int k = lane; k < mu * np; k += 32) BT[k] = T(0);
  __syncwarp();
  // B^T columns: entries of velocity rows in the seed (pressure) columns;
  // each row's entries are read eight at a time, all loads in flight
  for (int r = lane; r < mu; r += 32) {
    const int g = sdof[r];
    const int e1 = rowptr[g + 1];
    for (int e0 = rowptr[g]; e0 < e1; e0 += 8) {
      int cc[8];
      double vv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        cc[u] = e0 + u < e1 ? col[e0 + u] : -1;
        vv[u] = e0 + u < e1 ? Kval[e0 + u] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        for (int k = 0; k < np; ++k)
          if (sdof[mu + k] == cc[u]) BT[r * np + k] = T(vv[u]);
    }
  }
  const int nblk = shared ? 1 : dim;
  const bool tiled = i >= nsmall;  // one 32 x 32 tile
  const int blk = tiled ? kTileElems : padded_pk<T>(m);
  T* out = fac + foff[i];
  bool sing = false;
  for (int cb = 0; cb < nblk; ++cb) {
    __syncwarp();
    T row[MAXM];
#pragma unroll
    for (int j = 0; j < MAXM; ++j) row[j] = T(0);
    if (lane < m) {
#pragma unroll
      for (int j = 0; j < MAXM; ++j) Am[lane * L::kStride + j] = T(0);
      const int g = sdof[cb * m + lane];
      const int e1 = rowptr[g + 1];
      for (int e0 = rowptr[g]; e0 < e1; e0 += 8) {
        int cc[8];
        double vv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          cc[u] = e0 + u < e1 ? col[e0 + u] : -1;
          vv[u] = e0 + u < e1 ? Kval[e0 + u] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int pos = cc[u] >= 0 ? bsearch_int(sdof + cb * m, m, cc[u]) : -1;
          if (pos >= 0) Am[lane * L::kStride + pos] = T(vv[u]);
        }
      }
#pragma unroll
      for (int j = 0; j < MAXM; ++j) row[j] = Am[lane * L::kStride + j];
    }
    T dm = lane < m ? fabs(Am[lane * L::kStride + lane]) : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    // Gauss-Jordan inversion in registers; the block is SPD so no pivoting
#pragma unroll
    for (int k = 0; k < MAXM; ++k) {
      if (k < m) {
        __syncwarp();
        if (lane == k) {
#pragma unroll
          for (int j = 0; j < MAXM; ++j) prow[j] = row[j];
        }
        __syncwarp();
        T piv = prow[k];
        const bool bad = !(fabs(piv) > T(1e-12) * dm);
        if (bad) piv = T(1);  // keeps the arithmetic finite; the patch is flagged
        sing |= bad;
        const T p = T(1) / piv;
        const T f = lane == k ? T(1) - p : row[k] * p;
#pragma unroll
        for (int j = 0; j < MAXM; ++j) row[j] = fma(-f, prow[j], row[j]);
        row[k] = lane == k ? p : -f;
      }
    }
    // packed lower triangle of the (symmetrised) inverse
    __syncwarp();
    if (lane < m) {
#pragma unroll
      for (int j = 0; j < MAXM; ++j) Am[lane * L::kStride + j] = row[j];
    }
    __syncwarp();
    if (tiled) {
      for (int c = 0; c < 32; ++c)
        out[cb * blk + lane * 32 + (c ^ lane)] =
            lane < m && c < m ? T(0.5) * (Am[lane * L::kStride + c] + Am[c * L::kStride + lane]) : T(0);
    } else if (lane < m) {
      for (int b = 0; b <= lane; ++b)
        out[cb * blk + lane * (lane + 1) / 2 + b] = T(0.5) * (Am[lane * L::kStride + b] + Am[b * L::kStride + lane]);
    }
    // U rows of the components this block serves: U = A^-1 B^T
    const int c0 = shared ? 0 : cb, c1 = shared ? dim : cb + 1;
    if (lane < m)
      for (int c = c0; c < c1; ++c)
        for (int k = 0; k < np; ++k) {
          T s = T(0);
#pragma unroll
          for (int b = 0; b < MAXM; ++b)
            if (b < m) s = fma(row[b], BT[(c * m + b) * np + k], s);
          U[(c * m + lane) * np + k] = s;
        }
  }
  __syncwarp();
  // S = -B A^-1 B^T = -(B^T)^T U, np x np
  for (int kk = 0; kk < np * np; ++kk) {
    const int k = kk / np, k2 = kk - k * np;
    T s = T(0);
    for (int r = lane; r < mu; r += 32) s = fma(BT[r * np + k], U[r * np + k2], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) S[k * kMaxNp + k2] = -s;
  }
  T* Uout = out + nblk * blk;
  T* Sout = Uout + mu * np;
  for (int idx = lane; idx < mu * np; idx += 32) {
    const int r = idx / np, k = idx - r * np;
    Uout[k * mu + r] = U[r * np + k];
  }
  __syncwarp();
  if (lane == 0) {
    // S^-1 by Gauss-Jordan with partial pivoting (np <= 4)
    T M[kMaxNp][2 * kMaxNp];
    T smax = T(0);
    for (int a = 0; a < np; ++a)
      for (int b = 0; b < np; ++b) {
        M[a][b] = S[a * kMaxNp + b];
        M[a][np + b] = a == b ? T(1) : T(0);
        smax = fmax(smax, fabs(M[a][b]));
      }
    for (int k = 0; k < np && !sing; ++k) {
      int pr = k;
      for (int a = k + 1; a < np; ++a)
        if (fabs(M[a][k]) > fabs(M[pr][k])) pr = a;
      if (!(fabs(M[pr][k]) > T(1e-12) * smax)) { sing = true; break; }
      if (pr != k)
        for (int b = 0; b < 2 * np; ++b) { T t = M[k][b]; M[k][b] = M[pr][b]; M[pr][b] = t; }
      const T p = T(1) / M[k][k];
      for (int b = 0; b < 2 * np; ++b) M[k][b] *= p;
      for (int a = 0; a < np; ++a)
        if (a != k) {
          const T f = M[a][k];
          for (int b = 0; b < 2 * np; ++b) M[a][b] -= f * M[k][b];
        }
    }
    for (int a = 0; a < np; ++a)
      for (int b = 0; b < np; ++b) Sout[a * np + b] = sing ? T(0) : M[a][np + b];
    if (sing) atomicAdd(nsing, 1);
  }
}

template <typename T, int MAXM>
static cudaError_t launch_factor_warp(const DevPatches& p, const DevCSR& K, int start, int count, int* nsingular,
                                      cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  const size_t shm = kFacWarps * FacWarpSmem<T, MAXM>::bytes();
  const unsigned blocks = (unsigned)((count + kFacWarps - 1) / kFacWarps);
  SD_LAUNCH((k_vanka_factor_warp<T, MAXM>), blocks, kFacWarps * 32, shm, st, count, p.fac_list + start, p.dim, p.shared,
      p.ptr, p.dof, p.nvel, p.npres, p.foff, K.rowptr, K.col, K.v64, reinterpret_cast<T*>(p.fac), nsingular, p.nsmall);
  return cudaGetLastError();
}

int vanka_factor_warp_bin(int m) { return m <= 8 ? 0 : m <= 20 ? 1 : m <= 32 ? 2 : -1; }

size_t vanka_factor_smem(int dim, int max_m, int max_np, size_t elem, bool global_a) {
  return elem * ((global_a ? 0 : (size_t)max_m * max_m) + 2 * (size_t)dim * max_m * max_np + 2 * max_m +
                 kMaxNp * kMaxNp + 4) +
         sizeof(int) * ((size_t)dim * max_m + max_np) + 16;
}

// Factorise all patches: the warp-per-patch bins (m <= 32) lead the list;
// then, for FP32, the tensor-core blocked sweep, and for FP64 the
// CTA-per-patch Gauss-Jordan (blocks that fit in shared memory first, the
// rest in chunks of at most `fac_chunk` patches with the block in the global
// scratch gA).
template <typename T>
cudaError_t vanka_factor(const DevPatches& p, const DevCSR& K, int* nsingular, cudaStream_t st) {
  if (p.npatch == 0) return cudaSuccess;
  const int dm = p.dim;
  int start = 0;
  cudaError_t e0 = launch_factor_warp<T, 8>(p, K, start, p.nfac_warp[0], nsingular, st);
  if (e0 != cudaSuccess) return e0;
  start += p.nfac_warp[0];
  e0 = launch_factor_warp<T, 20>(p, K, start, p.nfac_warp[1], nsingular, st);
  if (e0 != cudaSuccess) return e0;
  start += p.nfac_warp[1];
  e0 = launch_factor_warp<T, 32>(p, K, start, p.nfac_warp[2], nsingular, st);
  if (e0 != cudaSuccess) return e0;
  start += p.nfac_warp[2];
  if constexpr (sizeof(T) == 4) {
    return vanka_factor_tc(p, K, start, nsingular, st);
  } else {
    if (p.nfac_smem > 0) {
      const size_t shm = vanka_factor_smem(dm, p.max_m_fac_smem, p.max_np, sizeof(T), false);
      SD_LAUNCH((k_vanka_factor<T>), p.nfac_smem, kFacThreads, shm, st, p.nfac_smem, p.fac_list + start, dm, p.shared, p.ptr,
                                                               p.dof, p.nvel, p.npres, p.foff, K.rowptr, K.col, K.v64,
                                                               reinterpret_cast<T*>(p.fac), nsingular,
                                                               p.max_m_fac_smem, p.max_np, (T*)nullptr, p.nsmall);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    start += p.nfac_smem;
    const int nglob = p.npatch - start;
    for (int c0 = 0; c0 < nglob; c0 += p.fac_chunk) {
      const int cnt = std::min(p.fac_chunk, nglob - c0);
      const size_t shm = vanka_factor_smem(dm, p.max_m, p.max_np, sizeof(T), true);
      SD_LAUNCH((k_vanka_factor<T>), cnt, kFacThreads, shm, st, cnt, p.fac_list + start + c0, dm, p.shared, p.ptr, p.dof,
                                                       p.nvel, p.npres, p.foff, K.rowptr, K.col, K.v64,
                                                       reinterpret_cast<T*>(p.fac), nsingular, p.max_m, p.max_np,
                                                       reinterpret_cast<T*>(p.fac_scratch), p.nsmall);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
}
template cudaError_t vanka_factor<float>(const DevPatches&, const DevCSR&, int*, cudaStream_t);
template cudaError_t vanka_factor<double>(const DevPatches&, const DevCSR&, int*, cudaStream_t);

// -------------------------------------------------------------- apply
// Copy n elements of T from global (16-byte aligned) to shared memory with
// 16-byte streaming loads (evict-first: the factors are read once per sweep
// and must not push the level vectors and index maps out of L2).
template <typename T>
__device__ __forceinline__ void group_copy(T* __restrict__ dst, const T* __restrict__ src, int n, int lane, int nl) {
  constexpr int V = 16 / sizeof(T);
  const int nv = n / V;
  const int4* s4 = reinterpret_cast<const int4*>(src);
  int4* d4 = reinterpret_cast<int4*>(dst);
  for (int k = lane; k < nv; k += nl) d4[k] = __ldcs(s4 + k);
  for (int k = nv * V + lane; k < n; k += nl) dst[k] = __ldcs(src + k);
}

// Persistent, warp-specialised patch solves.  Patches are stored bin by bin
// (by velocity DoFs per component), so the factor blocks, index lists and
// metadata of `tp` consecutive patches of a bin (a tile) are three
// contiguous ranges: one producer thread moves each tile into a
// shared-memory ring of `stages` buffers with 1D bulk copies
// (cp.async.bulk, evict-first in L2) completing on an mbarrier, while kNCW
// consumer warps solve the previous tiles.  A consumer warp gathers the
// right-hand side of its contiguous share of the tile into registers (all
// loads in flight), then LP lanes solve one patch, R matrix rows per lane
// (row a = l + i LP), so a warp holds 32 / LP patches at a time.
constexpr int kNCW = 4;

template <typename T, typename TR, int DIM, int NPM, int LP, int R>
__global__ void __launch_bounds__(32 * (kNCW + 1)) k_vanka_apply_tma(
    int pstart, int pcount, int ntiles, int tp, int stages, int fac_bytes, int dof_bytes, int rhs_elems, int shared,
    const int4* __restrict__ meta, const int* __restrict__ pptr, const int64_t* __restrict__ foff,
    const int* __restrict__ dof, const int* __restrict__ pdst, const T* __restrict__ fac, const TR* __restrict__ r,
    T* __restrict__ yp, int* __restrict__ err) {
  pdl_enter();
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + stages;
  // stage: factors | index lists | output positions | metadata
  const int stage_bytes = fac_bytes + 2 * dof_bytes + tp * 16;
  unsigned char* stage0 = smem + 128;
  T* rhsb = reinterpret_cast<T*>(stage0 + (size_t)stages * stage_bytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, kNCW);
    }
    mbar_fence_init();
  }
  __syncthreads();
  const int pend = pstart + pcount;
  if (warp == kNCW) {
    if (lane == 0) {
      const uint64_t pol = policy_evict_first();
      int k = 0, s = 0, round = 0;  // k = s + round * stages
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        if (round > 0 && !mbar_wait(empty + s, (round - 1) & 1)) {
          atomicOr(err, 1);
          break;
        }
        const int i0 = pstart + t * tp, i1 = min(i0 + tp, pend);
        const int64_t f0 = foff[i0], f1 = foff[i1];
        const int d0 = pptr[i0] & ~3, d1 = (pptr[i1] + 3) & ~3;
        const uint32_t fb = (uint32_t)((f1 - f0) * (int64_t)sizeof(T));
        const uint32_t db = (uint32_t)(d1 - d0) * 4u, mb = (uint32_t)(i1 - i0) * 16u;
        unsigned char* st = stage0 + (size_t)s * stage_bytes;
        mbar_expect_tx(full + s, fb + 2 * db + mb);
        bulk_g2s(st, fac + f0, fb, full + s, pol);
        bulk_g2s(st + fac_bytes, dof + d0, db, full + s, pol);
        bulk_g2s(st + fac_bytes + dof_bytes, pdst + d0, db, full + s, pol);
        bulk_g2s(st + fac_bytes + 2 * dof_bytes, meta + i0, mb, full + s, pol);
        if (++s == stages) {
          s = 0;
          ++round;
        }
      }
      // every copy issued has landed before this CTA may finish
      for (int kk = max(0, k - stages); kk < k; ++kk)
        if (!mbar_wait(full + (kk % stages), (kk / stages) & 1)) atomicOr(err, 4);
    }
    return;
  }
  constexpr int PPW = 32 / LP;  // patches a warp holds at a time (lanes past PPW*LP idle)
  T* myrhs = rhsb + (size_t)warp * rhs_elems;
  const int slot = lane / LP, l = lane % LP, gbase = slot * LP;
  const int nblk = shared ? 1 : DIM;
  int s = 0, round = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if (!mbar_wait(full + s, round & 1)) {
      atomicOr(err, 2);
      return;
    }
    const unsigned char* st = stage0 + (size_t)s * stage_bytes;
    const T* sfac = reinterpret_cast<const T*>(st);
    const int* sdof = reinterpret_cast<const int*>(st + fac_bytes);
    const int* sdst = reinterpret_cast<const int*>(st + fac_bytes + dof_bytes);
    const int4* smeta = reinterpret_cast<const int4*>(st + fac_bytes + 2 * dof_bytes);
    const int cnt = min(tp, pend - (pstart + t * tp));
    const int per = (cnt + kNCW - 1) / kNCW;
    const int j0 = min(warp * per, cnt), j1 = min(j0 + per, cnt);
    const int4 mf = smeta[0];
    const int a0 = mf.x & ~3;
    const int64_t ftile = (int64_t)(uint32_t)mf.z | ((int64_t)mf.w << 32);
    if (j0 < j1) {
      const int sb = smeta[j0].x;
      const int4 ml = smeta[j1 - 1];
      const int ns = ml.x + DIM * (ml.y & 0xffff) + (ml.y >> 16) - sb;
      constexpr int G = 4;
      for (int q0 = 0; q0 < ns; q0 += 32 * G) {
        TR v[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int q = q0 + g * 32 + lane;
          v[g] = q < ns ? r[sdof[sb - a0 + q]] : TR(0);
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const int q = q0 + g * 32 + lane;
          if (q < ns) myrhs[q] = T(v[g]);
        }
      }
      __syncwarp();
      for (int jb = j0; jb < j1; jb += PPW) {
        const int j = jb + slot;
        const bool valid = slot < PPW && j < j1;
        const int4 mt = smeta[valid ? j : jb];
        const int m = mt.y & 0xffff, np = mt.y >> 16, base = mt.x;
        const int mu = DIM * m;
        const int64_t fo = ((int64_t)(uint32_t)mt.z | ((int64_t)mt.w << 32)) - ftile;
        const int pkp = padded_pk<T>(m);
        const T* A = sfac + fo;
        const T* U = A + nblk * pkp;
        const T* Sv = U + mu * np;
        const T* bb = myrhs + (base - sb);
        int ca[R], ta[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
          ca[i] = min(l + i * LP, m - 1);
          ta[i] = ca[i] * (ca[i] + 1) / 2;
        }
        T acc[DIM][R];
#pragma unroll
        for (int c = 0; c < DIM; ++c)
#pragma unroll
          for (int i = 0; i < R; ++i) acc[c][i] = T(0);
        for (int blk = 0; blk < nblk; ++blk) {
          const T* Ab = A + blk * pkp;
          int tb = 0;
#pragma unroll 2
          for (int b = 0; b < m; ++b) {
            T va[R];
#pragma unroll
            for (int i = 0; i < R; ++i) va[i] = Ab[ca[i] >= b ? ta[i] + b : tb + ca[i]];
            if (shared) {
#pragma unroll
              for (int c = 0; c < DIM; ++c) {
                const T xv = bb[c * m + b];
#pragma unroll
                for (int i = 0; i < R; ++i) acc[c][i] += va[i] * xv;
              }
            } else {
              const T xv = bb[blk * m + b];
#pragma unroll
              for (int c = 0; c < DIM; ++c)
                if (c == blk)
#pragma unroll
                  for (int i = 0; i < R; ++i) acc[c][i] += va[i] * xv;
            }
            tb += b + 1;
          }
        }
        T tk[NPM], yk[NPM];
#pragma unroll
        for (int kk = 0; kk < NPM; ++kk) {
          T part = T(0);
          if (kk < np)
            for (int row = l; row < mu; row += LP) part += U[kk * mu + row] * bb[row];
          // fixed tree over the LP lanes of the group, then broadcast from its first lane
#pragma unroll
          for (int o = 1; o < LP; o <<= 1) {
            const T v = __shfl_down_sync(0xffffffffu, part, o);
            if ((l & (2 * o - 1)) == 0 && l + o < LP) part += v;
          }
          part = __shfl_sync(0xffffffffu, part, gbase < 32 ? gbase : 0);
          tk[kk] = kk < np ? bb[mu + kk] - part : T(0);
        }
#pragma unroll
        for (int kk = 0; kk < NPM; ++kk) {
          T v = T(0);
#pragma unroll
          for (int k2 = 0; k2 < NPM; ++k2)
            if (kk < np && k2 < np) v += Sv[kk * np + k2] * tk[k2];
          yk[kk] = v;
        }
        if (valid) {
#pragma unroll
          for (int c = 0; c < DIM; ++c)
#pragma unroll
            for (int i = 0; i < R; ++i) {
              const int a = l + i * LP;
              if (a < m) {
                T x = acc[c][i];
#pragma unroll
                for (int kk = 0; kk < NPM; ++kk)
                  if (kk < np) x -= U[kk * mu + c * m + a] * yk[kk];
                yp[sdst[base - a0 + c * m + a]] = x;
              }
            }
#pragma unroll
          for (int kk = 0; kk < NPM; ++kk)
            if (kk < np && l == kk) yp[sdst[base - a0 + mu + kk]] = yk[kk];
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + s);
    if (++s == stages) {
      s = 0;
      ++round;
    }
  }
}

// Bins (lanes per patch LP, rows per lane R): m <= 6 (6, 1), m <= 20 (10, 2),
// m <= 32 (16, 2), m <= 64 (32, 2), m <= 96 (32, 3).

template <typename T, typename TR, int DIM, int NPM, int LP, int R>
static cudaError_t launch_tma_bin(const DevPatches& p, const TmaBin& bn, const TR* r, T* yp, cudaStream_t st) {
  const size_t shm = 128 + (size_t)bn.stages * (bn.fac_bytes + 2 * bn.dof_bytes + bn.tp * 16) +
                     (size_t)kNCW * bn.rhs_elems * sizeof(T);
  SD_LAUNCH((k_vanka_apply_tma<T, TR, DIM, NPM, LP, R>), bn.grid, 32 * (kNCW + 1), shm, st, 
      bn.start, bn.count, bn.ntiles, bn.tp, bn.stages, bn.fac_bytes, bn.dof_bytes, bn.rhs_elems, p.shared, p.meta,
      p.ptr, p.foff, p.dof, p.pdst, reinterpret_cast<const T*>(p.fac), r, yp, p.err);
  return cudaGetLastError();
}

template <typename T, typename TR, int DIM, int NPM>
static cudaError_t launch_bin_np(const DevPatches& p, int b, const TR* r, T* yp, cudaStream_t st) {
  const TmaBin& bn = p.bins[b];
  switch (b) {
    case 0: return launch_tma_bin<T, TR, DIM, NPM, 6, 1>(p, bn, r, yp, st);
    case 1: return launch_tma_bin<T, TR, DIM, NPM, 10, 2>(p, bn, r, yp, st);
    case 2: return launch_tma_bin<T, TR, DIM, NPM, 16, 2>(p, bn, r, yp, st);
    case 3: return launch_tma_bin<T, TR, DIM, NPM, 32, 2>(p, bn, r, yp, st);
    default: return launch_tma_bin<T, TR, DIM, NPM, 32, 3>(p, bn, r, yp, st);
  }
}

template <typename T, typename TR>
static cudaError_t apply_tma_bin(const DevPatches& p, int b, const TR* r, T* yp, cudaStream_t st) {
  const TmaBin& bn = p.bins[b];
  if (bn.count == 0) return cudaSuccess;
  const bool one = bn.max_np <= 1;
  if (p.dim == 2) return one ? launch_bin_np<T, TR, 2, 1>(p, b, r, yp, st) : launch_bin_np<T, TR, 2, 4>(p, b, r, yp, st);
  return one ? launch_bin_np<T, TR, 3, 1>(p, b, r, yp, st) : launch_bin_np<T, TR, 3, 4>(p, b, r, yp, st);
}

cudaError_t vanka_apply_bin(const DevPatches& p, int b, const void* r, void* yp, bool fp32, cudaStream_t st) {
  if (b < 0 || b >= kTmaBins) return cudaErrorInvalidValue;
  if (fp32) return apply_tma_bin<float, float>(p, b, (const float*)r, (float*)yp, st);
  return apply_tma_bin<double, double>(p, b, (const double*)r, (double*)yp, st);
}

// Shared-memory bytes of a TMA bin's tile configuration.
size_t vanka_tma_smem(const DevPatches& p, const TmaBin& bn, size_t elem) {
  (void)p;
  return 128 + (size_t)bn.stages * (bn.fac_bytes + 2 * bn.dof_bytes + bn.tp * 16) +
         (size_t)kNCW * bn.rhs_elems * elem;
}

template <typename T, int DIM, int NPM>
static const void* tma_kernel_ptr(int b) {
  switch (b) {
    case 0: return (const void*)k_vanka_apply_tma<T, T, DIM, NPM, 6, 1>;
    case 1: return (const void*)k_vanka_apply_tma<T, T, DIM, NPM, 10, 2>;
    case 2: return (const void*)k_vanka_apply_tma<T, T, DIM, NPM, 16, 2>;
    case 3: return (const void*)k_vanka_apply_tma<T, T, DIM, NPM, 32, 2>;
    default: return (const void*)k_vanka_apply_tma<T, T, DIM, NPM, 32, 3>;
  }
}

static const void* tma_kernel(size_t elem, int dim, bool one, int b) {
  if (elem == 4) {
    if (dim == 2) return one ? tma_kernel_ptr<float, 2, 1>(b) : tma_kernel_ptr<float, 2, 4>(b);
    return one ? tma_kernel_ptr<float, 3, 1>(b) : tma_kernel_ptr<float, 3, 4>(b);
  }
  if (dim == 2) return one ? tma_kernel_ptr<double, 2, 1>(b) : tma_kernel_ptr<double, 2, 4>(b);
  return one ? tma_kernel_ptr<double, 3, 1>(b) : tma_kernel_ptr<double, 3, 4>(b);
}

int vanka_tma_blocks_per_sm(const DevPatches& p, const TmaBin& bn, int b, size_t elem) {
  int nb = 0;
  const void* k = tma_kernel(elem, p.dim, bn.max_np <= 1, b);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 32 * (kNCW + 1), vanka_tma_smem(p, bn, elem));
  return e == cudaSuccess ? nb : 0;
}

int vanka_tma_bin_of(int m) {
  return m <= 6 ? 0 : (m <= 20 ? 1 : (m <= 32 ? 2 : (m <= 64 ? 3 : (m <= 96 ? 4 : -1))));
}
int vanka_tma_bin_ppw(int b) { return b == 0 ? 5 : (b == 1 ? 3 : (b == 2 ? 2 : 1)); }

// The bins and the tiled patches are independent launches (disjoint patches
// and outputs).  With side streams they are forked off the main stream and
// joined back, so the small bins of a coarse level run side by side instead
// of one tail after another; captured into a graph they become parallel
// branches.
template <typename T, typename TR>
cudaError_t vanka_apply(const DevPatches& p, const TR* r, T* yp, cudaStream_t st, const ForkJoin* fj) {
  int parts[kTmaBins + 1], np = 0;
  if (p.nsmall > 0)
    for (int b = 0; b < kTmaBins; ++b)
      if (p.bins[b].count > 0) parts[np++] = b;
  if (p.nlarge > 0) parts[np++] = kTmaBins;
  const bool fork = fj != nullptr && np > 1 && np - 1 <= kForkMax;
  cudaError_t e = cudaSuccess;
  if (fork) e = cudaEventRecord(fj->fork, st);
  for (int k = 0; k < np && e == cudaSuccess; ++k) {
    cudaStream_t s = st;
    if (fork && k > 0) {
      s = fj->side[k - 1];
      e = cudaStreamWaitEvent(s, fj->fork, 0);
      if (e != cudaSuccess) break;
    }
    e = parts[k] == kTmaBins ? vanka_apply_tiles<T, TR>(p, r, yp, s) : apply_tma_bin<T, TR>(p, parts[k], r, yp, s);
    if (e == cudaSuccess && fork && k > 0) e = cudaEventRecord(fj->join[k - 1], s);
  }
  if (fork)
    for (int k = 1; k < np && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(st, fj->join[k - 1], 0);
  return e;
}
template cudaError_t vanka_apply<float, float>(const DevPatches&, const float*, float*, cudaStream_t, const ForkJoin*);
template cudaError_t vanka_apply<double, double>(const DevPatches&, const double*, double*, cudaStream_t,
                                                 const ForkJoin*);

// Allow every kernel with large dynamic shared memory the device's opt-in
// maximum once, so launches inside graph capture never need the attribute.
cudaError_t vanka_prepare_kernels() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  std::vector<const void*> ks = {
      (const void*)k_vanka_factor<float>, (const void*)k_vanka_factor<double>,
      (const void*)k_vanka_factor_warp<float, 8>, (const void*)k_vanka_factor_warp<float, 20>,
      (const void*)k_vanka_factor_warp<float, 32>, (const void*)k_vanka_factor_warp<double, 8>,
      (const void*)k_vanka_factor_warp<double, 20>, (const void*)k_vanka_factor_warp<double, 32>};
  for (size_t elem : {size_t(4), size_t(8)})
    for (int dim : {2, 3})
      for (bool one : {true, false})
        for (int b = 0; b < kTmaBins; ++b) ks.push_back(tma_kernel(elem, dim, one, b));
  for (const void* k : ks) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
  }
  return vanka_tiles_prepare_kernels(optin);
}

// -------------------------------------------------------------- scatter
// One thread per DoF: the apply stored the DoF's patch solutions
// contiguously (DoF-major, ascending original patch order), so the thread
// reads yp[tptr[j] .. tptr[j+1]) with four loads in flight, sums in that
// order and adds omega * sum / count.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_vanka_scatter(int64_t n, const int* __restrict__ tptr,
    const T* __restrict__ yp, T* __restrict__ x, T omega, const uint8_t* __restrict__ dir,
    const double* __restrict__ r64, double* __restrict__ out64, double* __restrict__ x64, T* __restrict__ xadd) {
  pdl_enter();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int b = tptr[j], e = tptr[j + 1];
  T s = T(0);
  for (int k = b; k < e; k += 4) {
    T v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = k + u < e ? yp[k + u] : T(0);
#pragma unroll
    for (int u = 0; u < 4; ++u) s += v[u];
  }
  const T upd = e > b ? omega * s / T(e - b) : T(0);
  if (MODE == 2) {
    out64[j] = dir[j] ? r64[j] : double(x[j] + upd);
    return;
  }
  const T xn = MODE == 0 ? upd : x[j] + upd;
  x[j] = xn;
  if (x64) x64[j] = double(xn);  // FP64 copy for the FP64 defect-correction residual
  if (xadd) xadd[j] += xn;       // the coarse correction of the level above (identity prolongation)
}

template <typename T>
cudaError_t vanka_scatter(const DevPatches& p, int64_t n, const T* yp, T* x, double omega, int mode,
                          const uint8_t* dir, const double* r64, double* out64, cudaStream_t st, double* x64,
                          T* xadd) {
  if (n == 0) return cudaSuccess;
  if (mode == 2 && xadd) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (mode == 0)
    SD_LAUNCH((k_vanka_scatter<T, 0>), blocks, 256, 0, st, n, p.tptr, yp, x, T(omega), dir, r64, out64, x64, xadd);
  else if (mode == 1)
    SD_LAUNCH((k_vanka_scatter<T, 1>), blocks, 256, 0, st, n, p.tptr, yp, x, T(omega), dir, r64, out64, x64, xadd);
  else
    SD_LAUNCH((k_vanka_scatter<T, 2>), blocks, 256, 0, st, n, p.tptr, yp, x, T(omega), dir, r64, out64, x64, xadd);
  return cudaGetLastError();
}
template cudaError_t vanka_scatter<float>(const DevPatches&, int64_t, const float*, float*, double, int,
                                          const uint8_t*, const double*, double*, cudaStream_t, double*, float*);
template cudaError_t vanka_scatter<double>(const DevPatches&, int64_t, const double*, double*, double, int,
                                           const uint8_t*, const double*, double*, cudaStream_t, double*, double*);

}  // namespace sd
