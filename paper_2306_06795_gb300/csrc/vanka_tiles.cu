// Large Vanka patches (Sec. 3.3.1; steps a5 and a6 for the patches outside
// the bulk-copy bins: coarse 3D levels with up to a few hundred velocity
// DoFs per component).  Their inverse velocity blocks are stored tiled
// (tiles.cuh).
//
// Factorisation, FP32: the SPD block A is inverted on chip by a blocked
// symmetric sweep (Gauss-Jordan elimination on 32 x 32 pivot blocks that
// keeps only the lower tiles).  For pivot block K with P = M_KK^-1:
//   X_i = M_iK P                      (i != K)
//   M_ij <- M_ij - X_i M_jK^T         (i >= j; i, j != K)
//   M_iK <- X_i,  M_KK <- -P
// and after the last pivot block M = -A^-1.  Both products are dense
// contractions and run on the tensor cores with the TF32 split
// x = x_hi + x_lo and three products per step, which keeps FP32 accuracy.
// Blocks of three tile rows (the 3D vertex patches) can use the
// 5th-generation tensor cores (stokes_params.factor_tcgen05): per pivot block, the stacked rows
// [M_iK]_{i != K} and P, then [X_i] and [M_jK], are staged in shared memory
// as K-major TF32 operands (hi and lo parts), one thread issues
// tcgen05.mma (M = 128, K = 8 per instruction) into a TMEM accumulator,
// completion arrives on an mbarrier and the four warps read the rows back
// with tcgen05.ld.  At these sizes (32 x 32 x 32 products) the staging, the
// two dependent MMA round trips per pivot block and the lower occupancy cost
// more than the faster products (C4: 22.5 ms against 17.7 ms), so the
// default, and every other block, uses mma.sync m16n8k8.  The 32 x 32 pivot
// inverse runs in the registers of one warp.
//
// Apply: a persistent kernel in which each consumer warp solves one patch
// at a time, fed by its own producer warp through a ring of bulk copies
// (index list, tiles, U and S^-1, output positions).  y_u = A^-1 b_u is
// accumulated tile by tile: a row sweep y_I += T b_J (lane = row) and, off
// the diagonal, a column sweep y_J += T^T b_I (lane = column), so every lane
// owns its rows of y and no cross-lane reductions are needed.
#include <algorithm>

#include "common.cuh"
#include "tiles.cuh"
#include "tma.cuh"
#include "umma.cuh"

namespace sd {

// =============================================================== factorise

// Factor-side tile layout: element (r, c) at r * 32 + (c ^ h(r)) with
// h(r) = ((r & 3) << 3) | (r & 4).  The m16n8k8 fragment reads (row from
// the lane's group g, column from its index t in the group, or the
// transpose of that) and the accumulator pairs hit 32 different banks.
__device__ __forceinline__ int fsw(int r, int c) { return (r << 5) + (c ^ (((r & 3) << 3) | (r & 4))); }

__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return u;
}

// x = hi + lo with both parts representable in TF32
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}

// d += a b for a 16 x 8 (row-major fragment) and b 8 x 8 (column fragment)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct FacTiles {
  float* M;  // lower tiles, (I, J) at I(I+1)/2 + J
  float* X;  // one tile per tile row
  __device__ __forceinline__ float* tile(int I, int J) const { return M + ((I * (I + 1) >> 1) + J) * kTileElems; }
  // element (r, c) of block (I, J) of the symmetric matrix
  __device__ __forceinline__ float get(int I, int J, int r, int c) const {
    return I >= J ? tile(I, J)[fsw(r, c)] : tile(J, I)[fsw(c, r)];
  }
};

// Rows r0 .. r0 + 15 of X_i = M_iK P (one warp).
__device__ __forceinline__ void tc_x_rows(const FacTiles& F, const float* P, int i, int K, int r0, int g, int t) {
  float acc[4][4];
#pragma unroll
  for (int n = 0; n < 4; ++n)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[n][q] = 0.f;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const int k0 = ks * 8;
    uint32_t ah[4], al[4];
    tf32_split(F.get(i, K, r0 + g, k0 + t), ah[0], al[0]);
    tf32_split(F.get(i, K, r0 + g + 8, k0 + t), ah[1], al[1]);
    tf32_split(F.get(i, K, r0 + g, k0 + t + 4), ah[2], al[2]);
    tf32_split(F.get(i, K, r0 + g + 8, k0 + t + 4), ah[3], al[3]);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      uint32_t bh0, bl0, bh1, bl1;
      tf32_split(P[fsw(k0 + t, n * 8 + g)], bh0, bl0);
      tf32_split(P[fsw(k0 + t + 4, n * 8 + g)], bh1, bl1);
      mma_tf32(acc[n], al, bh0, bh1);
      mma_tf32(acc[n], ah, bl0, bl1);
      mma_tf32(acc[n], ah, bh0, bh1);
    }
  }
  float* Xi = F.X + i * kTileElems;
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    *reinterpret_cast<float2*>(Xi + fsw(r0 + g, n * 8 + 2 * t)) = make_float2(acc[n][0], acc[n][1]);
    *reinterpret_cast<float2*>(Xi + fsw(r0 + g + 8, n * 8 + 2 * t)) = make_float2(acc[n][2], acc[n][3]);
  }
}

// Rows r0 .. r0 + 15 of M_ij -= X_i M_jK^T (one warp).
__device__ __forceinline__ void tc_update_rows(const FacTiles& F, int i, int j, int K, int r0, int g, int t) {
  float* C = F.tile(i, j);
  float acc[4][4];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const float2 u = *reinterpret_cast<const float2*>(C + fsw(r0 + g, n * 8 + 2 * t));
    const float2 w = *reinterpret_cast<const float2*>(C + fsw(r0 + g + 8, n * 8 + 2 * t));
    acc[n][0] = u.x;
    acc[n][1] = u.y;
    acc[n][2] = w.x;
    acc[n][3] = w.y;
  }
  const float* Xi = F.X + i * kTileElems;
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const int k0 = ks * 8;
    uint32_t ah[4], al[4];
    tf32_split(-Xi[fsw(r0 + g, k0 + t)], ah[0], al[0]);
    tf32_split(-Xi[fsw(r0 + g + 8, k0 + t)], ah[1], al[1]);
    tf32_split(-Xi[fsw(r0 + g, k0 + t + 4)], ah[2], al[2]);
    tf32_split(-Xi[fsw(r0 + g + 8, k0 + t + 4)], ah[3], al[3]);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      // B(k, n) = M_jK(n, k)
      uint32_t bh0, bl0, bh1, bl1;
      tf32_split(F.get(j, K, n * 8 + g, k0 + t), bh0, bl0);
      tf32_split(F.get(j, K, n * 8 + g, k0 + t + 4), bh1, bl1);
      mma_tf32(acc[n], al, bh0, bh1);
      mma_tf32(acc[n], ah, bl0, bl1);
      mma_tf32(acc[n], ah, bh0, bh1);
    }
  }
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    *reinterpret_cast<float2*>(C + fsw(r0 + g, n * 8 + 2 * t)) = make_float2(acc[n][0], acc[n][1]);
    *reinterpret_cast<float2*>(C + fsw(r0 + g + 8, n * 8 + 2 * t)) = make_float2(acc[n][2], acc[n][3]);
  }
}

// P = M_KK^-1 by Gauss-Jordan in the registers of one warp (lane r holds
// row r; the block is SPD, no pivoting) over its first kmax rows; writes P
// and M_KK <- -P.  Returns
// true when a pivot was not above thr (it is then replaced by 1, which keeps
// the arithmetic finite; the caller flags the patch).
__device__ bool tc_pivot_block(const FacTiles& F, float* P, float* prow, int K, int kmax, int lane, float thr) {
  float* D = F.tile(K, K);
  float row[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) row[c] = D[fsw(lane, c)];
  bool bad = false;
  float4* prow4 = reinterpret_cast<float4*>(prow);
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k >= kmax) break;  // padding rows (last tile row) stay decoupled; their entries are dropped
    if (lane == k) {
      float piv = row[k];
      if (!(fabsf(piv) > thr)) {
        piv = 1.f;
        bad = true;
      }
      const float ip = 1.f / piv;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = 4 * q + u == k ? ip : row[4 * q + u] * ip;
        prow4[q] = make_float4(v[0], v[1], v[2], v[3]);
      }
    }
    __syncwarp();
    const float f = row[k];
    const bool me = lane == k;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 p4 = prow4[q];
      const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = 4 * q + u;
        row[j] = me ? pv[u] : (j == k ? -f * pv[u] : fmaf(-f, pv[u], row[j]));
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    P[fsw(lane, c)] = row[c];
    D[fsw(lane, c)] = -row[c];
  }
  return __any_sync(0xffffffffu, bad);
}

// ------------------------------------------------ tcgen05 trailing products
// K-major TF32 operand of up to 128 rows and 32 K-columns: 8-row x 4-element
// (16-byte) core matrices, adjacent along K 128 bytes apart, 8-row groups
// 1024 bytes apart.  Offset of element (row, k) in floats, and its inverse
// (element e of the staging order, so consecutive threads write
// consecutive words).
__device__ __forceinline__ int kmaj_off(int row, int k) {
  return ((row >> 3) << 8) + ((k >> 2) << 5) + ((row & 7) << 2) + (k & 3);
}
__device__ __forceinline__ void kmaj_rc(int e, int& row, int& k) {
  row = ((e >> 8) << 3) + ((e >> 2) & 7);
  k = (((e >> 5) & 7) << 2) + (e & 3);
}
constexpr int kUmmaRowsA = 128;          // M of every MMA; rows past the operand are not read back
constexpr int kUmmaCols = 128;           // TMEM columns: X (32) and the trailing block (up to 64)
constexpr int kUmmaMaxRows = kUmmaMaxRowsFac;  // tile rows handled on tcgen05 (trailing block up to 64 columns)
constexpr uint32_t kUmmaLbo = 128, kUmmaSbo = 1024;

// Staging, 64 rows of 32 floats each, in the order A_hi, A_lo, B_hi, B_lo.
// An MMA reads 128 rows of A: from A_hi it reads A_hi and A_lo, from A_lo
// it reads A_lo and B_hi; the accumulator rows past the operand's (at most
// 64) rows are never read back, so the buffers need no padding.
constexpr int kUmmaStageRows = 64;
constexpr int kUmmaStageFloats = 4 * kUmmaStageRows * 32;

// D = A B^T for A (128 x 32) and B (N x 32) given as hi/lo TF32 parts: the
// three products lo*hi, hi*lo, hi*hi in four K-steps each, issued by the
// calling thread; completion arrives on bar.
__device__ __forceinline__ void umma_split_product(uint32_t d_tmem, const float* Ahi, const float* Alo,
                                                   const float* Bhi, const float* Blo, int N, uint64_t* bar) {
  tc_fence_after();
  const uint32_t idesc = idesc_tf32(kUmmaRowsA, N);
  const float* As[3] = {Alo, Ahi, Ahi};
  const float* Bs[3] = {Bhi, Blo, Bhi};
  uint32_t acc = 0;
  for (int q = 0; q < 3; ++q)
    for (int s = 0; s < 4; ++s) {  // K-step s covers k = 8s .. 8s + 7: two core matrices, 256 bytes
      const uint64_t ad = smem_desc_kmajor(As[q] + s * 64, kUmmaLbo, kUmmaSbo);
      const uint64_t bd = smem_desc_kmajor(Bs[q] + s * 64, kUmmaLbo, kUmmaSbo);
      umma_tf32(d_tmem, ad, bd, idesc, acc);
      acc = 1;
    }
  umma_commit(bar);
}

size_t vanka_factor_tc_smem(int dim, int rows, int max_np, bool global_tiles, bool umma) {
  const size_t ntl = (size_t)rows * (rows + 1) / 2;
  size_t f = (global_tiles ? 0 : (ntl + rows) * kTileElems) + kTileElems + 32 + 4 + kMaxNp * kMaxNp +
             2 * (size_t)dim * 32 * rows * max_np + (umma ? kUmmaStageFloats + 32 : 0);
  return f * sizeof(float) + sizeof(int) * ((size_t)dim * 32 * rows + max_np + 2 * (32 * (size_t)rows + 1)) + 16;
}

// Tensor-core factorisation CTA size: 128 threads for up to three tile rows
// (more CTAs per SM), 256 above.
constexpr int tc_threads(int rows) { return rows <= 3 ? 128 : 256; }

// One CTA of NTHR threads per patch.  `rows_max` is the tile-row capacity
// of the launch (the shared-memory layout); with gscr the tiles live in
// global scratch (rows_max tile rows per CTA).  Patches with storage id >=
// nsmall get the tiled block, the others the packed one.
template <int NTHR, bool UMMA>
__global__ void __launch_bounds__(NTHR, 512 / NTHR) k_vanka_factor_tc(int nlist, const int* __restrict__ list,
    int dim, int shared, const int* __restrict__ ptr, const int* __restrict__ dof, const int* __restrict__ nvel,
    const int* __restrict__ npres, const int64_t* __restrict__ foff, const int* __restrict__ rowptr,
    const int* __restrict__ col, const double* __restrict__ Kval, float* __restrict__ fac, int* nsing, int rows_max,
    int max_np, int nsmall, float* __restrict__ gscr, int* __restrict__ err) {
  pdl_enter();
  static_assert(!UMMA || NTHR == 128, "the tcgen05 path reads TMEM with one warpgroup");
  constexpr int NW = NTHR / 32;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if ((int)blockIdx.x >= nlist) return;
  const int i = list[blockIdx.x];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  const int base = ptr[i], m = nvel[i], np = npres[i];
  const int mu = dim * m, mt = mu + np;
  const int nT = tile_rows(m), nn = nT * 32, ntl = nT * (nT + 1) / 2;
  const int ntl_max = rows_max * (rows_max + 1) / 2;
  float* sp = reinterpret_cast<float*>(smem_raw);
  // tcgen05 staging (operands, then the mbarrier and the TMEM address)
  float* Ahi = sp;
  float* Alo = Ahi + kUmmaStageRows * 32;
  float* Bhi = Alo + kUmmaStageRows * 32;
  float* Blo = Bhi + kUmmaStageRows * 32;
  uint64_t* ubar = reinterpret_cast<uint64_t*>(Blo + kUmmaStageRows * 32);
  uint32_t* utaddr = reinterpret_cast<uint32_t*>(ubar + 1);
  if constexpr (UMMA) sp += kUmmaStageFloats + 32;
  uint32_t tmem = 0, uphase = 0;
  bool uok = true;
  if constexpr (UMMA) {
    if (warp == 0) tmem_alloc(utaddr, kUmmaCols);
    if (tid == 0) {
      mbar_init(ubar, 1);
      mbar_fence_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    tmem = *utaddr;
  }
  FacTiles F;
  if (gscr) {
    F.M = gscr + (size_t)blockIdx.x * (ntl_max + rows_max) * kTileElems;
  } else {
    F.M = sp;
    sp += (size_t)(ntl_max + rows_max) * kTileElems;
  }
  F.X = F.M + (size_t)ntl_max * kTileElems;
  float* P = sp;                    // [1024]
  float* prow = P + kTileElems;     // [32]
  float* misc = prow + 32;          // [0]: diagonal max, [1]: singular flag
  float* S = misc + 4;              // [kMaxNp^2]
  float* BT = S + kMaxNp * kMaxNp;  // [dim * 32 rows_max * max_np]
  float* U = BT + (size_t)dim * 32 * rows_max * max_np;
  int* sdof = reinterpret_cast<int*>(U + (size_t)dim * 32 * rows_max * max_np);
  int* rs = sdof + dim * 32 * rows_max + max_np;  // [32 rows_max + 1] first entry of each block row
  int* off = rs + 32 * rows_max + 1;             // [32 rows_max + 1] entry offsets of the block rows

  for (int k = tid; k < mt; k += NTHR) sdof[k] = dof[base + k];
  if (tid == 0) misc[1] = 0.f;
  __syncthreads();
  // B^T: entry (velocity row r, seed k) by binary search of the seed's
  // column in the row (columns ascending)
  for (int idx = tid; idx < mu * np; idx += NTHR) {
    const int r = idx / np, k = idx - r * np;
    const int key = sdof[mu + k], gr = sdof[r];
    int lo = rowptr[gr], hi = rowptr[gr + 1] - 1;
    float v = 0.f;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int x = col[mid];
      if (x == key) {
        v = float(Kval[mid]);
        break;
      }
      if (x < key) lo = mid + 1;
      else hi = mid - 1;
    }
    BT[r * np + k] = v;
  }
  const int nblk = shared ? 1 : dim;
  const bool tiled = i >= nsmall;
  const int64_t blk = tiled ? tiled_block_elems(m) : (int64_t)padded_pk<float>(m);
  float* out = fac + foff[i];
  for (int cb = 0; cb < nblk; ++cb) {
    __syncthreads();
    {
      float4* z = reinterpret_cast<float4*>(F.M);
      for (int e = tid; e < ntl * (kTileElems / 4); e += NTHR) z[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int a = tid; a < m; a += NTHR) {
      const int gr = sdof[cb * m + a];
      const int s0 = rowptr[gr];
      rs[a] = s0;
      off[a + 1] = rowptr[gr + 1] - s0;
    }
    if (tid == 0) off[0] = 0;
    __syncthreads();
    if (warp == 0) {  // running sum of the row lengths
      int carry = 0;
      for (int a0 = 1; a0 <= m; a0 += 32) {
        const int a = a0 + lane;
        int v = a <= m ? off[a] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int u = __shfl_up_sync(0xffffffffu, v, o);
          if (lane >= o) v += u;
        }
        if (a <= m) off[a] = v + carry;
        carry += __shfl_sync(0xffffffffu, v, 31);
      }
    }
    __syncthreads();
    // lower tiles of the block (diagonal tiles whole): the entries of the
    // block rows in one flat range, four loads in flight per thread
    const int E = off[m];
    for (int f0 = tid; f0 < E; f0 += 4 * NTHR) {
      int cc[4], ra[4];
      double vv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int f = f0 + u * NTHR;
        cc[u] = -1;
        ra[u] = 0;
        vv[u] = 0.0;
        if (f < E) {
          int lo = 0, hi = m - 1;  // block row a with off[a] <= f < off[a + 1]
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= f) lo = mid;
            else hi = mid - 1;
          }
          const int e = rs[lo] + f - off[lo];
          cc[u] = col[e];
          vv[u] = Kval[e];
          ra[u] = lo;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int pos = cc[u] >= 0 ? bsearch_int(sdof + cb * m, m, cc[u]) : -1;
        const int a = ra[u];
        if (pos >= 0 && (pos >> 5) <= (a >> 5)) F.tile(a >> 5, pos >> 5)[fsw(a & 31, pos & 31)] = float(vv[u]);
      }
    }
    __syncthreads();
    if (warp == 0) {
      // diagonal scale for the pivot test; the padding rows get a decoupled
      // diagonal of that size (their inverse is dropped on output)
      float dmax = 0.f;
      for (int a = lane; a < m; a += 32) dmax = fmaxf(dmax, fabsf(F.tile(a >> 5, a >> 5)[fsw(a & 31, a & 31)]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      const float pad = dmax > 0.f ? dmax : 1.f;
      for (int a = m + lane; a < nn; a += 32) F.tile(a >> 5, a >> 5)[fsw(a & 31, a & 31)] = pad;
      if (lane == 0) misc[0] = dmax;
    }
    __syncthreads();
    const float thr = 1e-12f * misc[0];
    for (int K = 0; K < nT; ++K) {
      if (warp == 0) {
        const bool bad = tc_pivot_block(F, P, prow, K, min(32, m - 32 * K), lane, thr);
        if (bad && lane == 0) misc[1] = 1.f;
      }
      __syncthreads();
      const int nr = nT - 1;
      if constexpr (UMMA) {
        if (nr > 0 && uok) {
          // pass 1: X = [M_iK]_{i != K} P  (rows 32 ii + r of A are row r of M_{i2,K})
          for (int e = tid; e < nr * 32 * 32; e += NTHR) {
            int q, k;
            kmaj_rc(e, q, k);
            const int ii = q >> 5, i2 = ii < K ? ii : ii + 1;
            uint32_t h, l;
            tf32_split(F.get(i2, K, q & 31, k), h, l);
            Ahi[e] = __uint_as_float(h);
            Alo[e] = __uint_as_float(l);
          }
          for (int e = tid; e < 32 * 32; e += NTHR) {  // B(n, k) = P(k, n)
            int n, k;
            kmaj_rc(e, n, k);
            uint32_t h, l;
            tf32_split(P[fsw(k, n)], h, l);
            Bhi[e] = __uint_as_float(h);
            Blo[e] = __uint_as_float(l);
          }
          fence_async_smem();
          __syncthreads();
          if (tid == 0) umma_split_product(tmem, Ahi, Alo, Bhi, Blo, 32, ubar);
          if (!mbar_wait(ubar, uphase)) uok = false;
          uphase ^= 1;
          uok = __syncthreads_and(uok);
          if (uok) {
            tc_fence_after();
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16), v);
            const int q = 32 * warp + lane;
            if (q < nr * 32) {
              const int ii = q >> 5, i2 = ii < K ? ii : ii + 1;
              float* Xi = F.X + i2 * kTileElems;
#pragma unroll
              for (int c = 0; c < 32; ++c) Xi[fsw(q & 31, c)] = v[c];
            }
            tc_fence_before();
          }
          __syncthreads();
          // pass 2: D = [X_i] [M_jK]^T, then M_ij -= D on the lower tiles
          if (uok) {
            for (int e = tid; e < nr * 32 * 32; e += NTHR) {
              int q, k;
              kmaj_rc(e, q, k);
              const int ii = q >> 5, i2 = ii < K ? ii : ii + 1;
              uint32_t h, l;
              tf32_split(F.X[i2 * kTileElems + fsw(q & 31, k)], h, l);
              Ahi[e] = __uint_as_float(h);
              Alo[e] = __uint_as_float(l);
              tf32_split(F.get(i2, K, q & 31, k), h, l);  // row n = q of B: row of M_{j2,K}
              Bhi[e] = __uint_as_float(h);
              Blo[e] = __uint_as_float(l);
            }
            fence_async_smem();
            __syncthreads();
            if (tid == 0) umma_split_product(tmem + 32, Ahi, Alo, Bhi, Blo, nr * 32, ubar);
            if (!mbar_wait(ubar, uphase)) uok = false;
            uphase ^= 1;
            uok = __syncthreads_and(uok);
            if (uok) {
              tc_fence_after();
              const int q = 32 * warp + lane;
              const int ii = q >> 5, i2 = ii < K ? ii : ii + 1;
              for (int jj = 0; jj < nr; ++jj) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32 + 32 * jj, v);
                const int j2 = jj < K ? jj : jj + 1;
                if (q < nr * 32 && j2 <= i2) {
                  float* C = F.tile(i2, j2);
#pragma unroll
                  for (int c = 0; c < 32; ++c) C[fsw(q & 31, c)] -= v[c];
                }
              }
              tc_fence_before();
            }
            __syncthreads();
          }
        }
      } else {
        for (int it = warp; it < 2 * (nT - 1); it += NW) {
          const int ii = it >> 1, i2 = ii < K ? ii : ii + 1;
          tc_x_rows(F, P, i2, K, (it & 1) * 16, g, t);
        }
        __syncthreads();
        for (int it = warp; it < nr * (nr + 1); it += NW) {
          const int q = it >> 1;
          int ia = 0;
          while ((ia + 1) * (ia + 2) / 2 <= q) ++ia;
          const int ja = q - ia * (ia + 1) / 2;
          tc_update_rows(F, ia < K ? ia : ia + 1, ja < K ? ja : ja + 1, K, (it & 1) * 16, g, t);
        }
        __syncthreads();
      }
      for (int e = tid; e < nr * kTileElems; e += NTHR) {
        const int ii = e >> 10, i2 = ii < K ? ii : ii + 1;
        const int r = (e >> 5) & 31, c = e & 31;
        const float x = F.X[i2 * kTileElems + fsw(r, c)];
        if (i2 > K) F.tile(i2, K)[fsw(r, c)] = x;
        else F.tile(K, i2)[fsw(c, r)] = x;
      }
      __syncthreads();
    }
    // M = -A^-1: lower triangle (diagonal tiles symmetrised), tiled or packed
    float* ob = out + cb * blk;
    if (tiled) {
      for (int q = warp; q < ntl; q += NW) {
        int I = 0;
        while ((I + 1) * (I + 2) / 2 <= q) ++I;
        const int J = q - I * (I + 1) / 2;
        const float* Tq = F.M + (size_t)q * kTileElems;
        for (int e = lane; e < kTileElems; e += 32) {
          const int r = e >> 5, c = (e & 31) ^ r;
          float v = 0.f;
          if (I * 32 + r < m && J * 32 + c < m)
            v = I == J ? -0.5f * (Tq[fsw(r, c)] + Tq[fsw(c, r)]) : -Tq[fsw(r, c)];
          ob[(size_t)q * kTileElems + e] = v;
        }
      }
    } else {
      for (int a = tid; a < m; a += NTHR) {
        const int I = a >> 5, r = a & 31;
        for (int b = 0; b <= a; ++b) {
          const int J = b >> 5, c = b & 31;
          const float* Tq = F.tile(I, J);
          ob[a * (a + 1) / 2 + b] = I == J ? -0.5f * (Tq[fsw(r, c)] + Tq[fsw(c, r)]) : -Tq[fsw(r, c)];
        }
      }
    }
    // U rows of the components this block serves: U = A^-1 B^T, one thread
    // per (row, component)
    const int c0 = shared ? 0 : cb, c1 = shared ? dim : cb + 1;
    for (int idx = tid; idx < m * (c1 - c0); idx += NTHR) {
      const int q = idx / m, a = idx - q * m, cc = c0 + q;
      float acc[kMaxNp];
#pragma unroll
      for (int k = 0; k < kMaxNp; ++k) acc[k] = 0.f;
      const int I = a >> 5, r = a & 31;
      const float* bt = BT + (size_t)cc * m * np;
      for (int b = 0; b < m; ++b) {
        const int J = b >> 5, c = b & 31;
        const float v = -(I >= J ? F.tile(I, J)[fsw(r, c)] : F.tile(J, I)[fsw(c, r)]);
#pragma unroll
        for (int k = 0; k < kMaxNp; ++k)
          if (k < np) acc[k] = fmaf(v, bt[b * np + k], acc[k]);
      }
#pragma unroll
      for (int k = 0; k < kMaxNp; ++k)
        if (k < np) U[(cc * m + a) * np + k] = acc[k];
    }
  }
  __syncthreads();
  // S = -B A^-1 B^T (np x np), one warp per entry
  for (int kk = warp; kk < np * np; kk += NW) {
    const int k = kk / np, k2 = kk - k * np;
    float s = 0.f;
    for (int r = lane; r < mu; r += 32) s = fmaf(BT[r * np + k], U[r * np + k2], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) S[k * kMaxNp + k2] = -s;
  }
  __syncthreads();
  float* Uout = out + nblk * blk;
  float* Sout = Uout + mu * np;
  for (int idx = tid; idx < mu * np; idx += NTHR) {
    const int r = idx / np, k = idx - r * np;
    Uout[k * mu + r] = U[r * np + k];
  }
  if (tid == 0) {
    // S^-1 by Gauss-Jordan with partial pivoting (np <= 4)
    float Mx[kMaxNp][2 * kMaxNp];
    float smax = 0.f;
    for (int a = 0; a < np; ++a)
      for (int b = 0; b < np; ++b) {
        Mx[a][b] = S[a * kMaxNp + b];
        Mx[a][np + b] = a == b ? 1.f : 0.f;
        smax = fmaxf(smax, fabsf(Mx[a][b]));
      }
    bool sing = misc[1] != 0.f;
    for (int k = 0; k < np && !sing; ++k) {
      int pr = k;
      for (int a = k + 1; a < np; ++a)
        if (fabsf(Mx[a][k]) > fabsf(Mx[pr][k])) pr = a;
      if (!(fabsf(Mx[pr][k]) > 1e-12f * smax)) {
        sing = true;
        break;
      }
      if (pr != k)
        for (int b = 0; b < 2 * np; ++b) {
          const float tmp = Mx[k][b];
          Mx[k][b] = Mx[pr][b];
          Mx[pr][b] = tmp;
        }
      const float p = 1.f / Mx[k][k];
      for (int b = 0; b < 2 * np; ++b) Mx[k][b] *= p;
      for (int a = 0; a < np; ++a)
        if (a != k) {
          const float f = Mx[a][k];
          for (int b = 0; b < 2 * np; ++b) Mx[a][b] -= f * Mx[k][b];
        }
    }
    for (int a = 0; a < np; ++a)
      for (int b = 0; b < np; ++b) Sout[a * np + b] = sing ? 0.f : Mx[a][np + b];
    if (sing) atomicAdd(nsing, 1);
  }
  if constexpr (UMMA) {
    // an MMA wait that ran out: the factors are unusable (flag for the
    // host); wait once more, boundedly, for the MMAs in flight before the
    // tensor memory is released
    if (!uok) {
      if (tid == 0) atomicOr(err, 32);
      mbar_wait(ubar, uphase ^ 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kUmmaCols);
  }
}

// Launches: the patches after `start` in the factorisation list, grouped by
// tile rows nT = 1..8 (tiles in shared memory, one launch per group sized
// for it), then the rest with the tiles in global scratch.
template <int NTHR, bool UMMA>
static cudaError_t launch_factor_tc(const DevPatches& p, const DevCSR& K, const int* list, int cnt, int rows,
                                    float* gscr, int* nsingular, cudaStream_t st) {
  const size_t shm = vanka_factor_tc_smem(p.dim, rows, p.max_np, gscr != nullptr, UMMA);
  SD_LAUNCH((k_vanka_factor_tc<NTHR, UMMA>), cnt, NTHR, shm, st, cnt, list, p.dim, p.shared, p.ptr, p.dof, p.nvel,
            p.npres, p.foff, K.rowptr, K.col, K.v64, reinterpret_cast<float*>(p.fac), nsingular, rows, p.max_np,
            p.nsmall, gscr, p.err);
  return cudaGetLastError();
}

cudaError_t vanka_factor_tc(const DevPatches& p, const DevCSR& K, int start, int* nsingular, cudaStream_t st) {
  for (int rows = 1; rows <= kTcMaxSmemRows; ++rows) {
    const int cnt = p.nfac_tc[rows];
    if (cnt == 0) continue;
    const cudaError_t e =
        p.tcgen05 && rows >= kUmmaMinRows && rows <= kUmmaMaxRows
            ? launch_factor_tc<128, true>(p, K, p.fac_list + start, cnt, rows, nullptr, nsingular, st)
        : tc_threads(rows) == 128
            ? launch_factor_tc<128, false>(p, K, p.fac_list + start, cnt, rows, nullptr, nsingular, st)
            : launch_factor_tc<256, false>(p, K, p.fac_list + start, cnt, rows, nullptr, nsingular, st);
    if (e != cudaSuccess) return e;
    start += cnt;
  }
  const int nglob = p.npatch - start;
  for (int c0 = 0; c0 < nglob; c0 += p.fac_chunk) {
    const int cnt = std::min(p.fac_chunk, nglob - c0);
    const cudaError_t e = launch_factor_tc<256, false>(p, K, p.fac_list + start + c0, cnt, p.tc_glob_rows,
                                                reinterpret_cast<float*>(p.fac_scratch), nsingular, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// =================================================================== apply
constexpr int kTilePairs = 4;  // consumer / producer warp pairs per CTA
constexpr int kTileBarBytes = 1024;

// node vectors of b and y: stride 4 (3D) or 2 (2D) elements per node
template <int DIM>
struct NodeStride {
  static constexpr int v = DIM == 3 ? 4 : 2;
};

// v[k] = p[c0 + k], k < NC, for a node vector p
template <typename T, int NC, int BS>
__device__ __forceinline__ void load_node(const T* p, int c0, T (&v)[NC]) {
  if constexpr (NC == 3 && sizeof(T) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
  } else if constexpr (NC == 2 && sizeof(T) == 4) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x;
    v[1] = q.y;
  } else if constexpr (NC >= 2 && sizeof(T) == 8) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x;
    v[1] = q.y;
    if constexpr (NC == 3) v[2] = p[2];
  } else {
#pragma unroll
    for (int k = 0; k < NC; ++k) v[k] = p[c0 + k];
  }
}

// One tile of the lower tiled block: y_I += T b_J (lane = row) and, for an
// off-diagonal tile, y_J += T^T b_I (lane = column); components c0 ..
// c0 + NC - 1 of the node vectors.
template <typename T, int NC, int BS>
__device__ __forceinline__ void tile_sweeps(const T* __restrict__ tl, const T* __restrict__ bv, T* __restrict__ yv,
                                            int I, int J, int c0, int lane) {
  T acc[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) acc[k] = T(0);
  const T* bj = bv + (size_t)J * 32 * BS;
  const int rb = lane * 33;  // lane * 32 + (c ^ lane) == (lane * 33) ^ c
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    const T a = tl[rb ^ c];
    T b[NC];
    load_node<T, NC, BS>(bj + c * BS, c0, b);
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = fma(a, b[k], acc[k]);
  }
  T* yi = yv + (size_t)(I * 32 + lane) * BS + c0;
#pragma unroll
  for (int k = 0; k < NC; ++k) yi[k] += acc[k];
  if (I == J) return;
#pragma unroll
  for (int k = 0; k < NC; ++k) acc[k] = T(0);
  const T* bi = bv + (size_t)I * 32 * BS;
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const T a = tl[(r * 33) ^ lane];
    T b[NC];
    load_node<T, NC, BS>(bi + r * BS, c0, b);
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = fma(a, b[k], acc[k]);
  }
  T* yj = yv + (size_t)(J * 32 + lane) * BS + c0;
#pragma unroll
  for (int k = 0; k < NC; ++k) yj[k] += acc[k];
}

// Chunks of one patch, in ring order: index list (16-byte aligned window),
// nblk * nT(nT+1)/2 tiles, U | S^-1 in pieces of one tile, output positions
// (aligned window).
__device__ __forceinline__ int tiles_patch_chunks(int m, int np, int dim, int nblk) {
  const int nT = tile_rows(m);
  const int L = dim * m * np + np * np;
  return 1 + nblk * nT * (nT + 1) / 2 + (L + kTileElems - 1) / kTileElems + 1;
}

template <typename T, typename TR, int DIM, int NPM>
__global__ void __launch_bounds__(64 * kTilePairs, 2) k_vanka_apply_tiles(int nlist, const int* __restrict__ list,
    int stages, int nodes, int shared, const int* __restrict__ ptr, const int* __restrict__ nvel,
    const int* __restrict__ npres, const int64_t* __restrict__ foff, const int* __restrict__ dof,
    const int* __restrict__ pdst, const T* __restrict__ fac, const TR* __restrict__ r, T* __restrict__ yp,
    int* __restrict__ err) {
  pdl_enter();
  constexpr int BS = NodeStride<DIM>::v;
  extern __shared__ __align__(128) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = warp >> 1;
  const bool producer = (warp & 1) != 0;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem) + (size_t)pair * 2 * stages;
  uint64_t* empty = full + stages;
  T* ring = reinterpret_cast<T*>(smem + kTileBarBytes) + (size_t)pair * stages * kTileElems;
  T* bv = reinterpret_cast<T*>(smem + kTileBarBytes) + (size_t)kTilePairs * stages * kTileElems +
          (size_t)pair * 2 * nodes * BS;
  T* yv = bv + (size_t)nodes * BS;
  if (threadIdx.x == 0) {
    uint64_t* b0 = reinterpret_cast<uint64_t*>(smem);
    for (int s = 0; s < kTilePairs * 2 * stages; ++s) mbar_init(b0 + s, 1);
    mbar_fence_init();
  }
  __syncthreads();
  const int nblk = shared ? 1 : DIM;
  const int G = gridDim.x * kTilePairs;
  const int first = blockIdx.x * kTilePairs + pair;
  if (producer) {
    if (lane == 0) {
      const uint64_t pol = policy_evict_first();
      int k = 0;  // chunks issued
      bool ok = true;
      for (int q = first; q < nlist && ok; q += G) {
        const int i = list[q];
        const int m = nvel[i], np = npres[i], base = ptr[i];
        const int mt = DIM * m + np;
        const int ntile = nblk * (tile_rows(m) * (tile_rows(m) + 1) / 2);
        const int L = DIM * m * np + np * np;
        const int nch = tiles_patch_chunks(m, np, DIM, nblk);
        const int64_t f0 = foff[i];
        const int d0 = base & ~3, d1 = (base + mt + 3) & ~3;
        for (int c = 0; c < nch; ++c) {
          const int s = k % stages;
          if (k >= stages && !mbar_wait(empty + s, ((k / stages) - 1) & 1)) {
            atomicOr(err, 1);
            ok = false;
            break;
          }
          T* dst = ring + (size_t)s * kTileElems;
          const void* src;
          uint32_t bytes;
          if (c == 0 || c == nch - 1) {
            src = (c == 0 ? dof : pdst) + d0;
            bytes = (uint32_t)(d1 - d0) * 4u;
          } else if (c <= ntile) {
            src = fac + f0 + (int64_t)(c - 1) * kTileElems;
            bytes = kTileElems * sizeof(T);
          } else {
            const int e0 = (c - 1 - ntile) * kTileElems;
            src = fac + f0 + (int64_t)ntile * kTileElems + e0;
            bytes = (uint32_t)(((size_t)min(kTileElems, L - e0) * sizeof(T) + 15) & ~(size_t)15);
          }
          mbar_expect_tx(full + s, bytes);
          bulk_g2s(dst, src, bytes, full + s, pol);
          ++k;
        }
      }
      // every copy issued has landed before this CTA may finish
      for (int kk = max(0, k - stages); kk < k; ++kk)
        if (!mbar_wait(full + (kk % stages), (kk / stages) & 1)) atomicOr(err, 4);
    }
    return;
  }
  int k = 0;  // chunks consumed
  for (int q = first; q < nlist; q += G) {
    const int i = list[q];
    const int m = nvel[i], np = npres[i], base = ptr[i];
    const int nT = tile_rows(m), nn = nT * 32;
    const int mu = DIM * m;
    const int doff = base & 3;
    // index list -> gathered right-hand side (zero on the padding nodes)
    if (!mbar_wait(full + k % stages, (k / stages) & 1)) {
      atomicOr(err, 2);
      return;
    }
    const int* sdof = reinterpret_cast<const int*>(ring + (size_t)(k % stages) * kTileElems) + doff;
    constexpr int GB = 4;
    for (int a0 = 0; a0 < nn; a0 += 32 * GB) {
      TR v[GB][DIM];
#pragma unroll
      for (int gb = 0; gb < GB; ++gb)
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          const int a = a0 + gb * 32 + lane;
          v[gb][c] = a < m ? r[sdof[c * m + a]] : TR(0);
        }
#pragma unroll
      for (int gb = 0; gb < GB; ++gb) {
        const int a = a0 + gb * 32 + lane;
        if (a < nn)
#pragma unroll
          for (int c = 0; c < BS; ++c) {
            bv[(size_t)a * BS + c] = c < DIM ? T(v[gb][c < DIM ? c : 0]) : T(0);
            yv[(size_t)a * BS + c] = T(0);
          }
      }
    }
    T bp[NPM];
#pragma unroll
    for (int kk = 0; kk < NPM; ++kk) bp[kk] = kk < np ? T(r[sdof[mu + kk]]) : T(0);
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + k % stages);
    ++k;
    // y_u = A^-1 b_u, tile by tile
    for (int cb = 0; cb < nblk; ++cb)
      for (int I = 0; I < nT; ++I)
        for (int J = 0; J <= I; ++J) {
          const int s = k % stages;
          if (!mbar_wait(full + s, (k / stages) & 1)) {
            atomicOr(err, 2);
            return;
          }
          const T* tl = ring + (size_t)s * kTileElems;
          if (shared) tile_sweeps<T, DIM, BS>(tl, bv, yv, I, J, 0, lane);
          else tile_sweeps<T, 1, BS>(tl, bv, yv, I, J, cb, lane);
          __syncwarp();
          if (lane == 0) mbar_arrive(empty + s);
          ++k;
        }
    // U | S^-1 and the output positions, all resident at once
    const int L = mu * np + np * np;
    const int nus = (L + kTileElems - 1) / kTileElems;
    for (int c = 0; c <= nus; ++c)
      if (!mbar_wait(full + (k + c) % stages, ((k + c) / stages) & 1)) {
        atomicOr(err, 2);
        return;
      }
    // element e of U | S^-1 (pieces of one tile in consecutive ring slots)
    const int ku = k;
    const auto usv = [ring, ku, stages](int e) -> T {
      return ring[(size_t)((ku + (e >> 10)) % stages) * kTileElems + (e & 1023)];
    };
    const int* sdst = reinterpret_cast<const int*>(ring + (size_t)((k + nus) % stages) * kTileElems) + doff;
    T yk[NPM];
    {
      T tk[NPM];
#pragma unroll
      for (int kk = 0; kk < NPM; ++kk) {
        T part = T(0);
        if (kk < np)
          for (int c = 0; c < DIM; ++c)
            for (int a = lane; a < m; a += 32) part += usv(kk * mu + c * m + a) * bv[(size_t)a * BS + c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        tk[kk] = kk < np ? bp[kk] - part : T(0);
      }
#pragma unroll
      for (int kk = 0; kk < NPM; ++kk) {
        T v = T(0);
#pragma unroll
        for (int k2 = 0; k2 < NPM; ++k2)
          if (kk < np && k2 < np) v += usv(mu * np + kk * np + k2) * tk[k2];
        yk[kk] = v;
      }
    }
    for (int c = 0; c < DIM; ++c)
      for (int a = lane; a < m; a += 32) {
        T x = yv[(size_t)a * BS + c];
#pragma unroll
        for (int kk = 0; kk < NPM; ++kk)
          if (kk < np) x -= usv(kk * mu + c * m + a) * yk[kk];
        yp[sdst[c * m + a]] = x;
      }
#pragma unroll
    for (int kk = 0; kk < NPM; ++kk)
      if (kk < np && lane == kk) yp[sdst[mu + kk]] = yk[kk];
    __syncwarp();
    if (lane == 0)
      for (int c = 0; c <= nus; ++c) mbar_arrive(empty + (k + c) % stages);
    k += nus + 1;
  }
}

size_t vanka_tiles_smem(int stages, int nodes, int dim, size_t elem) {
  const int bs = dim == 3 ? 4 : 2;
  return kTileBarBytes + elem * ((size_t)kTilePairs * stages * kTileElems + (size_t)kTilePairs * 2 * nodes * bs);
}

template <typename T, int DIM, int NPM>
static const void* tiles_kernel() {
  return (const void*)k_vanka_apply_tiles<T, T, DIM, NPM>;
}

static const void* tiles_kernel_of(size_t elem, int dim, bool one) {
  if (elem == 4) {
    if (dim == 2) return one ? tiles_kernel<float, 2, 1>() : tiles_kernel<float, 2, kMaxNp>();
    return one ? tiles_kernel<float, 3, 1>() : tiles_kernel<float, 3, kMaxNp>();
  }
  if (dim == 2) return one ? tiles_kernel<double, 2, 1>() : tiles_kernel<double, 2, kMaxNp>();
  return one ? tiles_kernel<double, 3, 1>() : tiles_kernel<double, 3, kMaxNp>();
}

int vanka_tiles_blocks_per_sm(int stages, int nodes, int dim, int np_max, size_t elem) {
  int nb = 0;
  const void* k = tiles_kernel_of(elem, dim, np_max <= 1);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 64 * kTilePairs,
                                                                vanka_tiles_smem(stages, nodes, dim, elem));
  return e == cudaSuccess ? nb : 0;
}

template <typename T, typename TR>
cudaError_t vanka_apply_tiles(const DevPatches& p, const TR* r, T* yp, cudaStream_t st) {
  if (p.nlarge == 0) return cudaSuccess;
  const size_t shm = vanka_tiles_smem(p.tiles_stages, p.tiles_nodes, p.dim, sizeof(T));
  const bool one = p.max_np <= 1;
#define SD_TILES_LAUNCH(D, NP)                                                                                     \
  SD_LAUNCH((k_vanka_apply_tiles<T, TR, D, NP>), p.tiles_grid, 64 * kTilePairs, shm, st,                                    \
      p.nlarge, p.large, p.tiles_stages, p.tiles_nodes, p.shared, p.ptr, p.nvel, p.npres, p.foff, p.dof, p.pdst,   \
      reinterpret_cast<const T*>(p.fac), r, yp, p.err)
  if (p.dim == 2) {
    if (one) SD_TILES_LAUNCH(2, 1);
    else SD_TILES_LAUNCH(2, kMaxNp);
  } else {
    if (one) SD_TILES_LAUNCH(3, 1);
    else SD_TILES_LAUNCH(3, kMaxNp);
  }
#undef SD_TILES_LAUNCH
  return cudaGetLastError();
}
template cudaError_t vanka_apply_tiles<float, float>(const DevPatches&, const float*, float*, cudaStream_t);
template cudaError_t vanka_apply_tiles<double, double>(const DevPatches&, const double*, double*, cudaStream_t);

cudaError_t vanka_tiles_prepare_kernels(int optin) {
  const void* ks[] = {(const void*)k_vanka_factor_tc<128, false>, (const void*)k_vanka_factor_tc<256, false>,
                      (const void*)k_vanka_factor_tc<128, true>,
                      tiles_kernel_of(4, 2, true),      tiles_kernel_of(4, 2, false),
                      tiles_kernel_of(4, 3, true),      tiles_kernel_of(4, 3, false), tiles_kernel_of(8, 2, true),
                      tiles_kernel_of(8, 2, false),     tiles_kernel_of(8, 3, true), tiles_kernel_of(8, 3, false)};
  for (const void* k : ks) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sd
