// The coarse tail of the V-cycle in one CTA.  On the last, tiny levels of
// the hierarchy (a few thousand DoFs) every step of Eq. TG-operator (Vanka
// sweeps, residuals, R_l, P_l, the coarsest bordered solve) is far too
// small to fill the GPU, and a separate launch per step costs more than
// the step itself.  One block of 1024 threads runs all of them in order,
// separated by block barriers; the data of these levels stays in L2.  The
// arithmetic is the level-by-level path's (same patch solves, same
// summation orders).
#include "common.cuh"

namespace sd {

namespace {

template <typename T>
__device__ void t_spmv(const TailCSR& A, const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ y,
                       int mode) {
  const T* val = reinterpret_cast<const T*>(A.val);
  for (int r = threadIdx.x; r < A.nrows; r += blockDim.x) {
    T s = T(0);
    for (int k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) s += val[k] * x[A.col[k]];
    if (mode == SPMV_SET) y[r] = s;
    else if (mode == SPMV_RES) y[r] = b[r] - s;
    else y[r] += s;
  }
}

__device__ __forceinline__ int t_packed(int a, int b) { return a >= b ? a * (a + 1) / 2 + b : b * (b + 1) / 2 + a; }

template <typename T>
__device__ __forceinline__ int t_padded_pk(int m) {
  constexpr int V = 16 / sizeof(T);
  return (m * (m + 1) / 2 + V - 1) / V * V;
}

// Patch solves of one level, one warp per patch, rows a = lane + 32 q (m <= 128);
// outputs at their DoF-major positions.
template <typename T>
__device__ void t_apply(const TailLevel& L, const T* __restrict__ rhs, T* __restrict__ yp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const T* fac = reinterpret_cast<const T*>(L.fac);
  const int dim = L.dim;
  const int nblk = L.shared ? 1 : dim;
  for (int i = warp; i < L.npatch; i += nw) {
    const int base = L.ptr[i], m = L.nvel[i], np = L.npres[i];
    const int mu = dim * m;
    const T* A = fac + L.foff[i];
    const int pkp = t_padded_pk<T>(m);
    const T* U = A + nblk * pkp;
    const T* S = U + mu * np;
    const int* dof = L.dof + base;
    const int* dst = L.pdst + base;
    T acc[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[c][q] = T(0);
    for (int c = 0; c < dim; ++c) {
      const T* Ab = A + (L.shared ? 0 : c) * pkp;
      for (int bb = 0; bb < m; ++bb) {
        const T xv = __ldg(rhs + __ldg(dof + c * m + bb));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int a = lane + 32 * q;
          if (a < m) acc[c][q] += Ab[t_packed(a, bb)] * xv;
        }
      }
    }
    T tk[4], yk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T part = T(0);
      if (k < np)
        for (int row = lane; row < mu; row += 32) part += U[k * mu + row] * rhs[dof[row]];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      tk[k] = k < np ? rhs[dof[mu + k]] - part : T(0);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      T v = T(0);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2)
        if (k < np && k2 < np) v += S[k * np + k2] * tk[k2];
      yk[k] = v;
    }
    for (int c = 0; c < dim; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = lane + 32 * q;
        if (a < m) {
          T x = acc[c][q];
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (k < np) x -= U[k * mu + c * m + a] * yk[k];
          yp[dst[c * m + a]] = x;
        }
      }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (k < np && lane == k) yp[dst[mu + k]] = yk[k];
  }
}

template <typename T>
__device__ void t_scatter(const TailLevel& L, const T* __restrict__ yp, T* __restrict__ x, int mode) {
  for (int j = threadIdx.x; j < L.n; j += blockDim.x) {
    const int b = L.tptr[j], e = L.tptr[j + 1];
    T s = T(0);
    for (int k = b; k < e; ++k) s += yp[k];
    const T upd = e > b ? T(L.omega) * s / T(e - b) : T(0);
    x[j] = mode == 0 ? upd : x[j] + upd;
  }
}

template <typename T>
__device__ void t_coarse(const TailLevel& L, const T* __restrict__ b, T* __restrict__ x) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = 0; k < L.nblocks; ++k) {
    const int n = L.bn[k], off = L.boff[k];
    const double* Kinv = L.Kinv + L.koff[k];
    for (int row = warp; row < n; row += nw) {
      double s = 0.0;
      for (int j = lane; j < n; j += 32) s += Kinv[(int64_t)row * n + j] * double(b[off + j]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) x[off + row] = T(s);
    }
  }
}

template <typename T>
__device__ void t_relax(const TailLevel& L, int nsweeps, bool zero_guess) {
  T* x = reinterpret_cast<T*>(L.x);
  const T* b = reinterpret_cast<const T*>(L.b);
  T* r = reinterpret_cast<T*>(L.r);
  T* yp = reinterpret_cast<T*>(L.yp);
  if (nsweeps == 0 && zero_guess) {
    for (int j = threadIdx.x; j < L.n; j += blockDim.x) x[j] = T(0);
    __syncthreads();
  }
  for (int s = 0; s < nsweeps; ++s) {
    if (s == 0 && zero_guess) {
      t_apply<T>(L, b, yp);
      __syncthreads();
      t_scatter<T>(L, yp, x, 0);
    } else {
      t_spmv<T>(L.K, x, b, r, SPMV_RES);
      __syncthreads();
      t_apply<T>(L, r, yp);
      __syncthreads();
      t_scatter<T>(L, yp, x, 1);
    }
    __syncthreads();
  }
}

}  // namespace

// Levels l0 .. l0+nl-1 of the V-cycle (input lv[0].b, output lv[0].x): the
// recursion of the level-by-level path unrolled into a down and an up pass.
template <typename T>
__global__ void __launch_bounds__(1024) k_tail(const TailLevel* __restrict__ lv, int nl, int nu1, int nu2) {
  for (int l = 0; l < nl - 1; ++l) {
    const TailLevel& L = lv[l];
    T* x = reinterpret_cast<T*>(L.x);
    const T* b = reinterpret_cast<const T*>(L.b);
    if (L.npatch > 0) {
      t_relax<T>(L, nu1, true);
    } else {
      for (int j = threadIdx.x; j < L.n; j += blockDim.x) x[j] = T(0);
      __syncthreads();
    }
    if (L.nblocks > 0) {
      t_coarse<T>(L, b, x);
      __syncthreads();
    }
    t_spmv<T>(L.K, x, b, reinterpret_cast<T*>(L.r), SPMV_RES);
    __syncthreads();
    t_spmv<T>(L.R, reinterpret_cast<const T*>(L.r), (const T*)nullptr, reinterpret_cast<T*>(lv[l + 1].b), SPMV_SET);
    __syncthreads();
  }
  {
    const TailLevel& C = lv[nl - 1];
    t_coarse<T>(C, reinterpret_cast<const T*>(C.b), reinterpret_cast<T*>(C.x));
    __syncthreads();
  }
  for (int l = nl - 2; l >= 0; --l) {
    const TailLevel& L = lv[l];
    t_spmv<T>(L.P, reinterpret_cast<const T*>(lv[l + 1].x), (const T*)nullptr, reinterpret_cast<T*>(L.x), SPMV_ADD);
    __syncthreads();
    if (L.npatch > 0) t_relax<T>(L, nu2, false);
  }
}

template <typename T>
cudaError_t tail_cycle(const TailLevel* lv, int nl, int nu1, int nu2, cudaStream_t st) {
  k_tail<T><<<1, 1024, 0, st>>>(lv, nl, nu1, nu2);
  return cudaGetLastError();
}
template cudaError_t tail_cycle<float>(const TailLevel*, int, int, int, cudaStream_t);
template cudaError_t tail_cycle<double>(const TailLevel*, int, int, int, cudaStream_t);

}  // namespace sd
