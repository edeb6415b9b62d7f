// Shared definitions of the CUDA solve path (device structures, launch
// wrappers).  Everything here is internal to libstokes_dcamg.so.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

namespace sd {

// Programmatic dependent launch.  A kernel launched by launch_pdl may be
// set up while the previous kernel of its stream is still finishing;
// pdl_enter(), the first statement of every kernel of the solve path, waits
// until that previous grid has completed and its writes are visible
// (griddepcontrol.wait), so the semantics stay those of plain stream order.
// No kernel triggers its dependents early (griddepcontrol.launch_dependents):
// measured on the C2 cycle, an early trigger made it slower (0.320 against
// 0.309 ms without PDL), the implicit trigger at grid exit faster (0.304 ms).
// Without a programmatic dependency the wait returns at once.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_wait() { pdl_enter(); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

// Launches kernel<<<grid, block, smem, st>>>(args...) with programmatic
// dependent launch from a function returning cudaError_t; returns the launch
// error.  A templated kernel name goes in parentheses.
#define SD_LAUNCH(kernel, grid, block, smem, st, ...)                                                   \
  do {                                                                                                  \
    cudaError_t e_launch_ = ::sd::launch_pdl(kernel, dim3(grid), dim3(block), (size_t)(smem), st, __VA_ARGS__); \
    if (e_launch_ != cudaSuccess) return e_launch_;                                                     \
  } while (0)

// CSR matrix on the device: int32 row pointers and columns (nnz < 2^31),
// FP64 values and, for an FP32 cycle, an FP32 copy of the values.
constexpr int kStreamNnz = 2048, kStreamRows = 256;

struct DevCSR {
  int nrows = 0, ncols = 0;
  int64_t nnz = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* v64 = nullptr;
  float* v32 = nullptr;
  int tpr = 4;  // threads per row of the vector-CSR SpMV
  // row-block tiles of the stream SpMV: {first row, first entry, end row,
  // end entry}, at most kStreamRows rows and kStreamNnz entries each
  int stiles = 0;
  int4* tdesc = nullptr;
  // sliced ELLPACK copy (large operators): chunks of 32 rows, entry k of row
  // 32 c + i at soff[c] + 32 k + i; rows shorter than the chunk are padded
  int schunks = 0;              // 0: no sliced copy
  int64_t* soff = nullptr;      // [schunks+1]
  int* scol = nullptr;
  double* sv64 = nullptr;
  float* sv32 = nullptr;
};

// SpMV modes
enum { SPMV_SET = 0, SPMV_RES = 1, SPMV_ADD = 2, SPMV_SCALED_RES = 3 };

// y = A x (SET), y = b - A x (RES), y += A x (ADD),
// y = s(row) (b - A x) with s = s1 where kind[row] == 1 else s0 (SCALED_RES).
// Accumulation in TACC.  TA: value type, TX/TB/TY: vector types.
template <typename TA, typename TX, typename TB, typename TY, typename TACC>
cudaError_t spmv(const DevCSR& A, const TA* val, const TX* x, const TB* b, TY* y, int mode,
                 double s0, double s1, const uint8_t* kind, cudaStream_t st);

// y = R b - (R K) x: the restricted residual of a level with R K assembled
// (R and RK have the same rows; vector CSR, the wider of their TPRs).
template <typename T>
cudaError_t restrict_res(const DevCSR& R, const T* rval, const T* b, const DevCSR& RK, const T* rkval, const T* x,
                         T* y, cudaStream_t st);

// Side streams and events that let independent launches of one step run
// side by side: fork on the main stream, launch on the sides, join back.
constexpr int kForkMax = 6;
struct ForkJoin {
  cudaStream_t side[kForkMax] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kForkMax] = {};
};

// A bin of patches solved by the bulk-copy kernel: storage patches
// [start, start + count), all with m in the bin's range.
constexpr int kTmaBins = 5;
constexpr int kTcMaxSmemRows = 8;  // tensor-core factorisation keeps up to 8 x 8 tile rows on chip
struct TmaBin {
  int start = 0, count = 0, tp = 0, ntiles = 0, grid = 0, stages = 3;
  int fac_bytes = 0, dof_bytes = 0, rhs_elems = 0, max_np = 0;
};

// Vanka patch data of one level on the device.
struct DevPatches {
  int npatch = 0;
  int dim = 2;
  int* ptr = nullptr;     // [npatch+1] offsets into dof (int32)
  int* dof = nullptr;     // [ptr[npatch]]
  int* nvel = nullptr;    // [npatch] velocity DoFs per component
  int* npres = nullptr;   // [npatch]
  int64_t* foff = nullptr;  // [npatch] factor offsets (elements)
  int64_t fac_elems = 0;
  void* fac = nullptr;    // factors, float or double
  int shared = 1;         // one velocity block shared by all components
  int tcgen05 = 0;        // FP32 three-tile-row blocks: trailing products on tcgen05
  int* small = nullptr;   // storage ids of the patches in bulk-copy bins (packed blocks)
  int nsmall = 0;
  int* large = nullptr;   // storage ids of the rest (tiled blocks), by descending m
  int nlarge = 0;
  int max_m = 0, max_np = 0, max_m_large = 0;
  int* tptr = nullptr;    // [n+1] DoF j's patch solutions are yp[tptr[j] .. tptr[j+1])
  int* pdst = nullptr;    // [nslots + 8] position in yp of each patch-major slot (DoF-major,
                          // ascending original patch order within a DoF)
  int64_t nslots = 0;
  // bulk-copy bins (storage order: bins by m, then the CTA-per-patch rest)
  int4* meta = nullptr;   // [npatch] {ptr, m | np << 16, foff lo, foff hi}
  bool use_tma = false;
  TmaBin bins[kTmaBins];
  int* err = nullptr;     // device error flags of the pipelines
  // factorisation: patches whose block fits in shared memory first
  int* fac_list = nullptr;
  int nfac_warp[3] = {0, 0, 0};  // warp-per-patch bins m <= 8, 20, 32 (first in fac_list)
  // FP64: CTA-per-patch Gauss-Jordan, blocks in shared memory, then the rest
  int nfac_smem = 0, max_m_fac_smem = 0, fac_chunk = 256;
  // FP32: tensor-core blocked sweep, per tile-row count nT = 1..8 with the
  // tiles in shared memory, then the rest with the tiles in global scratch
  int nfac_tc[kTcMaxSmemRows + 1] = {};
  int tc_glob_rows = 0;         // largest nT of the global-scratch patches
  void* fac_scratch = nullptr;  // per-chunk scratch of the global-memory variants
  // apply of the large patches (tiled blocks): ring stages per warp, node
  // capacity (32 * largest nT) and persistent grid
  int tiles_stages = 0, tiles_nodes = 0, tiles_grid = 0;
};

size_t vanka_factor_smem(int dim, int max_m, int max_np, size_t elem, bool global_a);
size_t vanka_factor_tc_smem(int dim, int rows, int max_np, bool global_tiles, bool umma);
// Tile rows whose blocks may be factorised with tcgen05 products (the 3D
// vertex patches, m = 65), when the handle asks for it.
constexpr int kUmmaMinRows = 3, kUmmaMaxRowsFac = 3;
int vanka_factor_warp_bin(int m);  // 0, 1, 2 for m <= 8, 20, 32; -1 above
size_t vanka_tiles_smem(int stages, int nodes, int dim, size_t elem);
int vanka_tiles_blocks_per_sm(int stages, int nodes, int dim, int np_max, size_t elem);

}  // namespace sd
struct stokes_handle;
namespace sd {
struct VankaView {
  const DevPatches* pat;
  int64_t n;
  bool fp32;
  cudaStream_t st;
};
int vanka_level_view(stokes_handle* h, int l, VankaView* v);
int stream_join_in(stokes_handle* h);
int stream_join_out(stokes_handle* h);
int set_error(int code, const char* msg);

size_t vanka_tma_smem(const DevPatches& p, const TmaBin& bn, size_t elem);
cudaError_t vanka_prepare_kernels();
int vanka_tma_blocks_per_sm(const DevPatches& p, const TmaBin& bn, int b, size_t elem);
int vanka_tma_bin_of(int m);
int vanka_tma_bin_ppw(int b);
// one bulk-copy bin of the apply (timing by the autotuner)
cudaError_t vanka_apply_bin(const DevPatches& p, int b, const void* r, void* yp, bool fp32, cudaStream_t st);

template <typename T>
cudaError_t vanka_factor(const DevPatches& p, const DevCSR& K, int* nsingular, cudaStream_t st);
// FP32 factorisation of the CTA-per-patch patches (m > 32) on tensor cores
cudaError_t vanka_factor_tc(const DevPatches& p, const DevCSR& K, int start, int* nsingular, cudaStream_t st);
// patch solves of the large patches (tiled blocks)
template <typename T, typename TR>
cudaError_t vanka_apply_tiles(const DevPatches& p, const TR* r, T* yp, cudaStream_t st);
cudaError_t vanka_tiles_prepare_kernels(int optin);

// Patch solves of Eqs. vanka_fact1/2 for every patch: yp (patch-major) =
// K_i^-1 V_i r.
template <typename T, typename TR>
cudaError_t vanka_apply(const DevPatches& p, const TR* r, T* yp, cudaStream_t st, const ForkJoin* fj = nullptr);

// Weighted scatter of Eq. vanka: s_j = sum over the patch slots of DoF j in
// ascending patch order; mode 0: x_j = omega s_j / cnt_j; mode 1: x_j +=
// omega s_j / cnt_j; mode 2 (final level-0 output): out_j = dir_j ? r64_j :
// double(x_j + omega s_j / cnt_j).  With x64 (modes 0, 1) the new x is also
// written in FP64; with xadd (modes 0, 1) it is also added to xadd_j.
template <typename T>
cudaError_t vanka_scatter(const DevPatches& p, int64_t n, const T* yp, T* x, double omega, int mode,
                          const uint8_t* dir, const double* r64, double* out64, cudaStream_t st,
                          double* x64 = nullptr, T* xadd = nullptr);

// Elementwise helpers
template <typename TI, typename TO>
cudaError_t cast_copy(int64_t n, const TI* in, TO* out, cudaStream_t st);
template <typename T, typename TI>
cudaError_t axpy_into(int64_t n, double a, const TI* xin, T* y, cudaStream_t st);   // y += a x
template <typename T>
cudaError_t fill_zero(int64_t n, T* y, cudaStream_t st);
template <typename T>
cudaError_t diag_scale(int64_t n, const T* d, const T* u, T* z, cudaStream_t st);  // z = d .* u
// z[j] = dir[j] ? r64[j] : du[j] (j < nu); z[nu + i] = sp * dp[i] (i < np)
template <typename T>
cudaError_t btp_out(int64_t nu, int64_t np, const T* du, const T* dp, double sp, const uint8_t* dir,
                    const double* r64, double* z, cudaStream_t st);
// out_j = dir_j ? r64_j : double(x_j)
template <typename T>
cudaError_t finalize_out(int64_t n, const T* x, const uint8_t* dir, const double* r64, double* out, cudaStream_t st);
// Write (flush) a buffer larger than L2.
cudaError_t l2_flush(void* buf, size_t bytes, cudaStream_t st);

// Chebyshev semi-iteration pieces (Saad, Alg. 12.1), zero initial guess:
//   init:  r = mask ? s * (dinv ? dinv*b : b) : 0;  d = r / theta;  x = 0
//   step:  y = M w;  x += d;  r -= (dinv ? dinv*y : y);  d_out = alpha d + beta r
// (w = d for a plain operator; w = B^T d for the B B^T products of DLSC).
template <typename T>
cudaError_t cheb_init(int64_t n, const T* b, const T* dinv, const uint8_t* mask, uint8_t want, double s, double theta,
                      T* r, T* d, T* x, cudaStream_t st);
template <typename T>
cudaError_t cheb_step(const DevCSR& M, const T* val, const T* w, const T* dinv, T* x, T* r, const T* d_in, T* d_out,
                      double alpha, double beta, cudaStream_t st);
// The first step fused with the initialisation (no mask, no dinv):
//   d0 = (s / theta) b;  x = d0 (accumulate: x += d0);  r = s b - M d0;
//   d_out = alpha d0 + beta r
template <typename T>
cudaError_t cheb_first(const DevCSR& M, const T* val, const T* b, double s, double theta, T* x, T* r, T* d_out,
                       double alpha, double beta, bool accumulate, cudaStream_t st);
// out[rows[i]] = T(in[i])
template <typename TI, typename TO>
cudaError_t scatter_rows(int64_t n, const TI* in, const int* rows, TO* out, cudaStream_t st);

// Coarsest exact solve: for each block k, y[off_k + i] = sum_j Kinv_k[i][j] b[off_k + j]
// (Kinv_k: n_k x n_k leading block of the bordered inverse, FP64 row-major).
template <typename T>
cudaError_t coarse_solve(int nblocks, const int* boff, const int* bn, const int64_t* koff,
                         const double* Kinv, int max_n, const T* b, T* y, cudaStream_t st);

// Segmented deterministic reductions for FGMRES (FP64).  Rows are cut into
// chunks that never straddle a segment (instance).  partial[c*ldp + k] =
// sum_{rows of chunk c} V_k[row] * w[row] for k < ncols (V_k = V + k*ldv).
cudaError_t multidot_partial(int nchunks, const int64_t* cbeg, const int64_t* cend, int ncols,
                             const double* V, int64_t ldv, const double* w, double* partial, int ldp,
                             cudaStream_t st);
// h[s*ldh + k] = (accumulate ? h : 0) + sum over chunks of segment s (in order) of partial
cudaError_t multidot_finish(int nseg, const int* sc_beg, const int* sc_end, int ncols,
                            const double* partial, int ldp, double* h, int ldh, int accumulate,
                            cudaStream_t st);
// w[row] += sign * sum_k coef[seg(row)*ldh + k] * V_k[row]
cudaError_t multiaxpy(int nchunks, const int64_t* cbeg, const int64_t* cend, const int* cseg, int ncols,
                      const double* V, int64_t ldv, const double* coef, int ldh, double sign, double* w,
                      cudaStream_t st);
// Device Galerkin product Kc = P^T K P (galerkin.cu); host CSR in, host
// arrays out (new[]); status 1: a row over the per-row product capacity.
cudaError_t galerkin_rap(int n, const int64_t* krp, const int* kcol, const double* kval, int nc, const int64_t* prp,
                         const int* pcol, const double* pval, cudaStream_t st, int* status, int64_t** crp,
                         int** ccol, double** cval, int64_t* cnnz);
// Further device steps of the AMG setup (Alg. 1): host arrays in, host arrays
// out (allocated with new[]).
cudaError_t sa_strength(int n, const int64_t* rp, const int* col, const double* val, double theta, cudaStream_t st,
                        int64_t** srp, int** scol, double** sval, int64_t* snnz);
cudaError_t sa_tentative(int n, const int* agg, int na, const double* B, cudaStream_t st, int64_t** trp, int** tcol,
                         double** tval, int64_t* tnnz, double* Bc);
cudaError_t sa_smooth(int n, const int64_t* arp, const int* acol, const double* aval, int nc, const int64_t* trp,
                      const int* tcol, const double* tval, double omega, cudaStream_t st, int* status,
                      int64_t** prp, int** pcol, double** pval, int64_t* pnnz);
cudaError_t vanka_patch_lists(int n, const int64_t* rp, const int* col, const double* val, const int64_t* hoff, int dim,
                              double rel_tol, cudaStream_t st, int* status, int* npatch, int64_t** hptr, int** hdof,
                              int** hnvel, int** hnpres);

// Krylov-wrapped relaxation (krylov.cu).  Rows of a level cut into chunks
// that never straddle an instance; sbeg/send: chunk range of each instance.
constexpr int kKrMaxSteps = 4;  // inner FGMRES steps per relaxation call
struct KrChunks {
  int n = 0;
  int64_t* beg = nullptr;
  int64_t* end = nullptr;
  int* seg = nullptr;
  int* sbeg = nullptr;
  int* send = nullptr;
};
struct KrCols {
  int c[kKrMaxSteps];  // scalar slots of a multi-column reduction
};
// n_0 = ||r||^2 per instance (scalar slot 0); u0 receives r unless u0 == r
template <typename T>
cudaError_t kr_norm0(const KrChunks& ch, const T* r, T* u0, double* partial, int ldp, int* cnt, double* S, int lds,
                     cudaStream_t st);
// c_ij = (w, U_i), i <= j, per instance
template <typename T>
cudaError_t kr_project(const KrChunks& ch, int j, int k, const T* U, int64_t ldu, const T* w, double* partial,
                       int ldp, int* cnt, double* S, int lds, cudaStream_t st);
// w -= sum_{i<=j} (c_ij / n_i) U_i, then n_{j+1} = ||w||^2, per instance
template <typename T>
cudaError_t kr_orthogonalise(const KrChunks& ch, int j, int k, const T* U, int64_t ldu, T* w, double* partial,
                             int ldp, int* cnt, double* S, int lds, cudaStream_t st);
// least squares from the scalars, then x = (set ? 0 : x) + Z coef; optional
// FP64 copy and level-0 output
template <typename T>
cudaError_t kr_update(const KrChunks& ch, int k, const T* Z, int64_t ldz, const double* S, int lds, T* x, int set,
                      double* x64, const uint8_t* dir, const double* r64, double* out64, cudaStream_t st);

// Device state of restarted FGMRES, per instance.
struct FgState {
  double* H;      // [ninst][(m+1)*m], row i column j at i*m + j
  double* cs;     // [ninst][m]
  double* sn;     // [ninst][m]
  double* g;      // [ninst][m+1]
  double* bnorm;  // [ninst]
  double* scale;  // [ninst] factor of the next Krylov vector (0 when stopped)
  double* y;      // [ninst][ldh] coefficients of x += Z y
  int* run;       // [ninst]
  int* its;       // [ninst]
  int* kcol;      // [ninst]
  int* err;       // [1] non-finite value seen
  int* stat;      // [m+1] any instance running after step j (index m: after the start)
};
cudaError_t fg_start(int ninst, int m, const FgState& st, const double* h, int ldh, double rtol, int maxit, int first,
                     cudaStream_t s);
cudaError_t fg_update(int ninst, int m, int j, const FgState& st, const double* h1, const double* h2, int ldh,
                      double rtol, int maxit, cudaStream_t s);
cudaError_t fg_solve(int ninst, int m, const FgState& st, int ldh, cudaStream_t s);
// Fused classical Gram-Schmidt passes of Arnoldi step j = nc - 1 for
// nc <= kArMaxCols columns over the chunks ch (fgmres.cu):
//   ar_dots:             h[s*ldh + k] = V_k . w per instance s (zero_flag, when
//                        given, is set to 0 first)
//   ar_axpy_dots:        w -= V coef_s, then h = V^T w
//   ar_axpy_norm_update: w -= V h2_s, then the Givens update of column j from
//                        h1, h2 and ||w||^2 (stat[j] collects the running flags)
constexpr int kArMaxCols = 32;
cudaError_t ar_dots(const KrChunks& ch, int nc, const double* V, int64_t ldv, const double* w, double* partial,
                    int ldp, int* cnt, double* h, int ldh, int* zero_flag, cudaStream_t s);
cudaError_t ar_axpy_dots(const KrChunks& ch, int nc, const double* V, int64_t ldv, const double* coef, int ldh,
                         double* w, double* partial, int ldp, int* cnt, double* h, cudaStream_t s);
cudaError_t ar_axpy_norm_update(const KrChunks& ch, int nc, const double* V, int64_t ldv, const double* h1,
                                const double* h2, int ldh, double* w, double* partial, int ldp, int* cnt, int m, int j,
                                const FgState& st, double rtol, int maxit, cudaStream_t s);
// out[row] = in[row] * f[seg(row)] (0 when f is 0); out32, when given,
// receives the same values rounded to FP32
cudaError_t seg_mul(int nchunks, const int64_t* cbeg, const int64_t* cend, const int* cseg, const double* in,
                    double* out, const double* f, cudaStream_t s, float* out32 = nullptr);

// out[row] = in[row] * scale_inv(seg)  where scale_inv = (den[seg*ldd + kd] > 0 && active[seg]) ? 1/den : 0
cudaError_t seg_scale(int nchunks, const int64_t* cbeg, const int64_t* cend, const int* cseg,
                      const double* in, double* out, const double* den, int ldd, int kd,
                      const int* active, int sqrt_den, cudaStream_t st);

}  // namespace sd
