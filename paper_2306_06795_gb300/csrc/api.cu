// Host orchestration of the solve phase behind the C ABI of
// include/stokes_dcamg.h: device setup of the hierarchy, batched patch
// factorisation, the defect-correction cycle (Eq. TG-operator-full around
// the Galerkin V-cycle of Eq. TG-operator), its CUDA-graph capture, and
// FP64 flexible GMRES with per-instance scalars (Sec. 4).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "common.cuh"
#include "stokes_dcamg.h"
#include "tiles.cuh"

using namespace sd;

static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                                       \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess)                                                                             \
      return fail(e_ == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA,                  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                                 \
  } while (0)

#define TRY(call)                \
  do {                           \
    int rc_ = (call);            \
    if (rc_ != STOKES_OK) return rc_; \
  } while (0)

namespace {

struct HostCSR {
  int nrows = 0, ncols = 0;
  std::vector<int> rowptr{0};
  std::vector<int> col;
  std::vector<double> val;
};

struct CoarseSet {
  int nblocks = 0, max_n = 0;
  int* boff = nullptr;
  int* bn = nullptr;
  int64_t* koff = nullptr;
  double* Kinv = nullptr;
  int64_t kinv_elems = 0;
};

// DLSC relaxation data of one level (Sec. 3.3.2, Alg. 2): the velocity
// block A, B and Mu^-1 B^T as level-sized CSRs (rows outside the block are
// empty), the row kinds and the Chebyshev bounds.  Mu = I on levels >= 1;
// on level 0 Mu = diag(Mu_diag): BT holds the rows of B^T scaled by 1/Mu
// and muinv (velocity rows 1/Mu, pressure rows 0) scales A's product in the
// pressure-correction right-hand side.
struct DLSCData {
  DevCSR A, B, BT;
  // p0 > 0: the level's rows are velocity rows [0, p0) then pressure rows
  // [p0, n) (one instance), and A, B, B^T hold only their nonempty rows:
  // A the velocity rows, B the pressure rows, B^T the velocity rows with
  // its columns counted from p0; the sweep works on the two row ranges
  int64_t p0 = 0;
  DevCSR S;                 // p0 > 0: S = B Mu^-1 B^T on the pressure rows (formed in FP64 at setup)
  bool pp_zero = false;     // K has no pressure-pressure entries on the relaxed rows
  DevCSR T;                 // p0 > 0: T = B Mu^-1 A Mu^-1 B^T on the pressure rows (setup, FP64)
  uint8_t* kind = nullptr;  // 0 velocity, 1 pressure, 2 rows not relaxed here
  double lamA = 0, lamS = 0;
  void* muinv = nullptr;    // level vector in the cycle precision, or nullptr (Mu = I)
  void* v[9] = {nullptr};   // res, v, q, dp, t1, t2, r, d0, d1
};

struct Level {
  int64_t n = 0;
  DevCSR K;
  bool hasP = false, Pident = false;
  DevCSR P, R;
  bool hasRK = false;  // R K assembled: the restricted residual is one launch
  DevCSR RK;
  bool has_patches = false;
  DevPatches pat;
  double omega = 1.0;
  int relax = STOKES_RELAX_VANKA;
  void* x = nullptr;
  void* b = nullptr;
  void* r = nullptr;
  void* yp = nullptr;
  void* ta = nullptr;  // scratch for stokes_level_op
  void* tb = nullptr;
  CoarseSet coarse;
  std::vector<int64_t> seg_off;  // per instance, -1 when absent
  bool dlsc = false;
  DLSCData dl;
  std::vector<int64_t> hfoff;  // host copies of the patch factor offsets and list pointers
  std::vector<int> hpptr;      // (bin re-tiling by the autotuner)
  // Krylov-wrapped relaxation (Sec. 3.3.1); jacobi: its inner
  // preconditioner is diag(K)^-1 instead of a Vanka sweep (BTP's SA cycles)
  bool krylov = false;
  bool jacobi = false;
  void* dinv = nullptr;
  int kmax = 0, lds = 0, ldp = 0;
  KrChunks kch;
  void* kV = nullptr;  // kmax + 1 level vectors
  void* kZ = nullptr;  // kmax level vectors
  double* kS = nullptr;       // per-instance scalars
  double* kpart = nullptr;    // chunk partials
  int* kcnt = nullptr;        // per-instance completion counters (0 between calls)
};

struct Ledger {
  bool count = false;
  double bytes = 0.0;
  int launches = 0;
};

}  // namespace

struct stokes_handle {
  int ninst = 0, dim = 2, disc = STOKES_TH, prec = STOKES_FP32, L = 0;
  // preconditioner: the DC cycle, or the block-triangular BTP (Sec. 4)
  int precond = STOKES_PRECOND_DC;
  std::string tune_report = "{}";  // autotuner choices (JSON)
  int btp_steps = 2;
  bool factor_tcgen05 = false;     // 3-tile-row FP32 patch blocks: tcgen05 trailing products
  std::vector<Level> btpA, btpM;  // SA hierarchies of A and of M_p / nu (TH)
  DevCSR btpB, btpMinv;           // B (pressure rows x velocity columns); SV exact mass inverse
  void* btp_tp = nullptr;         // level-0 pressure work vector
  int schedule = 0, nu1 = 1, nu2 = 1;
  double eta_u = 1.0, eta_p = 1.0;
  cudaStream_t st = nullptr;
  bool own_stream = false;     // created here: joined with the legacy default stream per call
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  ForkJoin fj;                 // side streams for independent launches of one step
  std::vector<Level> lv;
  std::vector<int> inst_levels;
  uint8_t* kind0 = nullptr;  // level 0: 0 velocity, 1 pressure, 2 Dirichlet
  int cheb_deg[3] = {3, 3, 6};
  int dlsc_sweeps = 2;
  // Scott-Vogelius restriction R0 = blockdiag(I, Mcg^-1 Pi^T M_dg)
  DevCSR R0v, R0q, Mcg;
  int64_t ncg = 0;
  int* prow1 = nullptr;      // level-1 row of each compressed pressure entry
  double* mdinv = nullptr;   // 1 / diag(Mcg)
  double* cv[5] = {nullptr}; // Chebyshev-Jacobi: rhs, x, r, d0, d1
  double* d0buf = nullptr;   // FP64 DC residual of level 0
  double* x0_64 = nullptr;   // FP64 copy of the level-0 iterate (FP32 cycle)
  double mcg_lo = 0.5, mcg_hi = 2.0;
  int mcg_deg = 32;
  uint8_t* dir0 = nullptr;   // level 0: 1 on Dirichlet rows
  bool factored = false;
  Ledger led;
  std::map<std::pair<const void*, void*>, cudaGraphExec_t> graphs;
  // FGMRES storage
  int krylov_m = 0;
  double* V = nullptr;
  double* Z = nullptr;
  double* w = nullptr;
  double* partial = nullptr;
  void* fold_x0 = nullptr;    // while the DC cycle runs level 1: x0, which level 1's last scatter adds x1 to
  bool folded = false;        // ... and whether it did
  bool r32_ready = false;     // the FP32 copy of the cycle input is already in lv[0].b (FGMRES steps)
  double* hd = nullptr;   // device h: [ninst][ldh]
  double* yd = nullptr;   // device coefficients [ninst][ldh]
  int* actd = nullptr;
  int ldh = 0, ldp = 0;
  int nchunks = 0;
  int64_t* cbeg = nullptr;
  int64_t* cend = nullptr;
  int* cseg = nullptr;
  int ndchunks = 0;  // larger chunks of the dot products
  int64_t* dbeg = nullptr;
  int64_t* dend = nullptr;
  int* sd_beg = nullptr;
  int* sd_end = nullptr;
  KrChunks arch;              // the dot-product chunks with their instances (fused Arnoldi passes)
  int* arcnt = nullptr;       // per-instance completion counters of the fused passes (0 between launches)
  void* flush = nullptr;
  size_t flush_bytes = 0;
  int64_t launches = 0;       // kernels launched so far
  FgState fg{};               // device-side FGMRES state
  int* hstat = nullptr;       // pinned: running flag after each Arnoldi step
  std::vector<cudaEvent_t> ev_iter;
  std::map<std::tuple<int, double, int>, cudaGraphExec_t> iter_graphs;
  int cycle_launches = -1;    // kernels in one DC cycle (from the ledger)
  std::vector<void*> allocs;
  std::vector<int*> err_flags;  // device error flags of every bulk-copy pipeline
  int* dsing = nullptr;         // singular-patch counter of the factorisation
};

// ------------------------------------------------------------- utilities
namespace {

template <typename T>
int dalloc(stokes_handle* h, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(e));
  h->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return STOKES_OK;
}

template <typename T>
int upload(stokes_handle* h, T** p, const std::vector<T>& v) {
  TRY(dalloc(h, p, v.size()));
  if (!v.empty()) CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return STOKES_OK;
}

int choose_tpr(int64_t nnz, int nrows) {
  const double mean = nrows ? double(nnz) / nrows : 0.0;
  if (mean <= 3) return 2;
  if (mean <= 6) return 4;
  if (mean <= 12) return 8;
  if (mean <= 24) return 16;
  return 32;
}

// Largest stored/nonzero ratio of a sliced-ELLPACK copy, and the fewest rows
// for one (smaller operators keep enough warps busy with vector CSR).
constexpr double kSellMaxPad = 1.25;
constexpr int kSellRows = 262144;
// Operators with kStreamMinRows <= rows < kSellRows use the row-block
// stream SpMV.
constexpr int kStreamMinRows = 32768;

int upload_csr(stokes_handle* h, DevCSR& d, const HostCSR& c, int sell_rows = kSellRows) {
  d.nrows = c.nrows;
  d.ncols = c.ncols;
  d.nnz = (int64_t)c.col.size();
  std::vector<int> rp(c.rowptr);
  std::vector<int> cl(c.col);
  std::vector<double> v(c.val);
  TRY(upload(h, &d.rowptr, rp));
  TRY(upload(h, &d.col, cl));
  TRY(upload(h, &d.v64, v));
  if (h->prec == STOKES_FP32) {
    std::vector<float> v32(v.begin(), v.end());
    TRY(upload(h, &d.v32, v32));
  }
  d.tpr = choose_tpr(d.nnz, d.nrows);
  int maxrow = 0;
  for (int i = 0; i < c.nrows; ++i) maxrow = std::max(maxrow, c.rowptr[i + 1] - c.rowptr[i]);
  // row-block tiles for the stream SpMV: mid-size operators, and large ones
  // whose row lengths vary too much for a sliced-ELLPACK copy
  auto stream_tiles = [&]() -> int {
    std::vector<int4> td;
    int r = 0;
    while (r < c.nrows) {
      int r1 = r;
      while (r1 < c.nrows && r1 - r < kStreamRows && c.rowptr[r1 + 1] - c.rowptr[r] <= kStreamNnz) ++r1;
      td.push_back(make_int4(r, c.rowptr[r], r1, c.rowptr[r1]));
      r = r1;
    }
    d.stiles = (int)td.size();
    TRY(upload(h, &d.tdesc, td));
    return STOKES_OK;
  };
  if (c.nrows >= kStreamMinRows && c.nrows < sell_rows && maxrow <= kStreamNnz) return stream_tiles();
  // sliced ELLPACK copy when the padding to the longest row of each chunk
  // of 32 rows stays small
  if (c.nrows >= sell_rows) {
    const int nch = (c.nrows + 31) / 32;
    std::vector<int64_t> off(nch + 1, 0);
    for (int ch = 0; ch < nch; ++ch) {
      int w = 0;
      for (int i = ch * 32; i < std::min(c.nrows, ch * 32 + 32); ++i) w = std::max(w, c.rowptr[i + 1] - c.rowptr[i]);
      off[ch + 1] = off[ch] + 32 * (int64_t)w;
    }
    if ((double)off[nch] <= kSellMaxPad * (double)std::max<int64_t>(d.nnz, 1)) {
      std::vector<int> scol(off[nch], -1);  // padding: column -1
      std::vector<double> sval(off[nch], 0.0);
      for (int i = 0; i < c.nrows; ++i) {
        const int64_t base = off[i / 32] + (i % 32);
        for (int k = c.rowptr[i]; k < c.rowptr[i + 1]; ++k) {
          scol[base + 32 * (int64_t)(k - c.rowptr[i])] = c.col[k];
          sval[base + 32 * (int64_t)(k - c.rowptr[i])] = c.val[k];
        }
      }
      TRY(upload(h, &d.soff, off));
      TRY(upload(h, &d.scol, scol));
      TRY(upload(h, &d.sv64, sval));
      if (h->prec == STOKES_FP32) {
        std::vector<float> s32(sval.begin(), sval.end());
        TRY(upload(h, &d.sv32, s32));
      }
      d.schunks = nch;
      return STOKES_OK;
    }
    if (maxrow <= kStreamNnz) return stream_tiles();
  }
  return STOKES_OK;
}

int check_csr(const stokes_csr* c, const char* what) {
  if (!c || c->nrows < 0 || c->ncols < 0 || c->nnz < 0 || (c->nnz > 0 && (!c->col || !c->val)) || !c->rowptr)
    return fail(STOKES_ERR_INVALID_ARG, std::string(what) + ": null or negative CSR fields");
  if (c->nnz >= (int64_t(1) << 31)) return fail(STOKES_ERR_INVALID_ARG, std::string(what) + ": nnz >= 2^31");
  if (c->rowptr[0] != 0 || c->rowptr[c->nrows] != c->nnz)
    return fail(STOKES_ERR_INVALID_ARG, std::string(what) + ": rowptr does not span nnz");
  for (int i = 0; i < c->nrows; ++i) {
    if (c->rowptr[i + 1] < c->rowptr[i]) return fail(STOKES_ERR_INVALID_ARG, std::string(what) + ": rowptr decreases");
    for (int64_t k = c->rowptr[i]; k < c->rowptr[i + 1]; ++k) {
      if (c->col[k] < 0 || c->col[k] >= c->ncols)
        return fail(STOKES_ERR_INVALID_ARG, std::string(what) + ": column index out of range");
      if (k > c->rowptr[i] && c->col[k] <= c->col[k - 1])
        return fail(STOKES_ERR_INVALID_ARG, std::string(what) + ": columns not sorted/unique");
      if (!std::isfinite(c->val[k])) return fail(STOKES_ERR_NAN, std::string(what) + ": non-finite value");
    }
  }
  return STOKES_OK;
}

// Append block (c) at (r0, c0) of the block-diagonal concatenation.
void append_block(HostCSR& out, const stokes_csr* c, int64_t c0) {
  for (int i = 0; i < c->nrows; ++i) {
    for (int64_t k = c->rowptr[i]; k < c->rowptr[i + 1]; ++k) {
      out.col.push_back((int)(c0 + c->col[k]));
      out.val.push_back(c->val[k]);
    }
    out.rowptr.push_back((int)out.col.size());
  }
}
void append_zero_rows(HostCSR& out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) out.rowptr.push_back((int)out.col.size());
}

HostCSR transpose(const HostCSR& a) {
  HostCSR t;
  t.nrows = a.ncols;
  t.ncols = a.nrows;
  t.rowptr.assign(a.ncols + 1, 0);
  for (int c : a.col) t.rowptr[c + 1]++;
  for (int i = 0; i < a.ncols; ++i) t.rowptr[i + 1] += t.rowptr[i];
  t.col.resize(a.col.size());
  t.val.resize(a.val.size());
  std::vector<int> pos(t.rowptr.begin(), t.rowptr.end() - 1);
  for (int i = 0; i < a.nrows; ++i)
    for (int k = a.rowptr[i]; k < a.rowptr[i + 1]; ++k) {
      const int p = pos[a.col[k]]++;
      t.col[p] = i;
      t.val[p] = a.val[k];
    }
  return t;
}

// X Y of two host CSRs (X's columns index Y's rows), row i scaled by rs[i]
// when given: FP64 sums in the order of X's row, then Y's row k; columns
// sorted.
HostCSR csr_product(const HostCSR& X, const HostCSR& Y, const double* rs) {
  HostCSR Z;
  Z.nrows = X.nrows;
  Z.ncols = Y.ncols;
  std::vector<double> acc(Y.ncols, 0.0);
  std::vector<int> mark(Y.ncols, -1), cols;
  for (int i = 0; i < X.nrows; ++i) {
    cols.clear();
    for (int e = X.rowptr[i]; e < X.rowptr[i + 1]; ++e) {
      const int k = X.col[e];
      const double xik = X.val[e];
      for (int f = Y.rowptr[k]; f < Y.rowptr[k + 1]; ++f) {
        const int j = Y.col[f];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = 0.0;
          cols.push_back(j);
        }
        acc[j] += xik * Y.val[f];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int j : cols) {
      Z.col.push_back(j);
      Z.val.push_back(rs ? rs[i] * acc[j] : acc[j]);
    }
    Z.rowptr.push_back((int)Z.col.size());
  }
  return Z;
}

bool is_identity(const stokes_csr* c) {
  if (c->nrows != c->ncols || c->nnz != c->nrows) return false;
  for (int i = 0; i < c->nrows; ++i)
    if (c->rowptr[i] != i || c->col[i] != i || c->val[i] != 1.0) return false;
  return true;
}

// Is K's velocity block of every component equal to component 0's (same
// pattern and values, shifted), so that patch blocks can be shared?
bool components_share_block(const stokes_csr* K, const int64_t* off, int dim) {
  const int64_t n0 = off[1] - off[0];
  for (int c = 1; c < dim; ++c) {
    if (off[c + 1] - off[c] != n0) return false;
    for (int64_t i = 0; i < n0; ++i) {
      const int64_t r0 = off[0] + i, rc = off[c] + i;
      // entries of each row inside its own component's column range
      std::vector<std::pair<int64_t, double>> a, b;
      for (int64_t k = K->rowptr[r0]; k < K->rowptr[r0 + 1]; ++k)
        if (K->col[k] >= off[0] && K->col[k] < off[1]) a.push_back({K->col[k] - off[0], K->val[k]});
      for (int64_t k = K->rowptr[rc]; k < K->rowptr[rc + 1]; ++k)
        if (K->col[k] >= off[c] && K->col[k] < off[c + 1]) b.push_back({K->col[k] - off[c], K->val[k]});
      if (a != b) return false;
    }
  }
  return true;
}

// Dense inverse of the bordered coarsest matrix [K n; n^T 0] by LU with
// partial pivoting (FP64); returns the leading n x n block row-major.
int bordered_inverse(const stokes_csr* K, const double* nullv, std::vector<double>& out) {
  const int n = K->nrows, nb = nullv ? n + 1 : n;  // no border: the plain inverse
  std::vector<double> M((size_t)nb * nb, 0.0), I((size_t)nb * nb, 0.0);
  for (int i = 0; i < n; ++i)
    for (int64_t k = K->rowptr[i]; k < K->rowptr[i + 1]; ++k) M[(size_t)i * nb + K->col[k]] = K->val[k];
  if (nullv)
    for (int i = 0; i < n; ++i) {
      M[(size_t)i * nb + n] = nullv[i];
      M[(size_t)n * nb + i] = nullv[i];
    }
  for (int i = 0; i < nb; ++i) I[(size_t)i * nb + i] = 1.0;
  double amax = 0.0;
  for (double v : M) amax = std::max(amax, std::fabs(v));
  for (int k = 0; k < nb; ++k) {
    int p = k;
    for (int i = k + 1; i < nb; ++i)
      if (std::fabs(M[(size_t)i * nb + k]) > std::fabs(M[(size_t)p * nb + k])) p = i;
    if (!(std::fabs(M[(size_t)p * nb + k]) > 1e-14 * amax))
      return fail(STOKES_ERR_SINGULAR_PATCH, "coarsest bordered matrix is singular");
    if (p != k)
      for (int j = 0; j < nb; ++j) {
        std::swap(M[(size_t)k * nb + j], M[(size_t)p * nb + j]);
        std::swap(I[(size_t)k * nb + j], I[(size_t)p * nb + j]);
      }
    const double piv = M[(size_t)k * nb + k];
    for (int i = k + 1; i < nb; ++i) {
      const double f = M[(size_t)i * nb + k] / piv;
      if (f == 0.0) continue;
      for (int j = k; j < nb; ++j) M[(size_t)i * nb + j] -= f * M[(size_t)k * nb + j];
      for (int j = 0; j < nb; ++j) I[(size_t)i * nb + j] -= f * I[(size_t)k * nb + j];
    }
  }
  // back substitution for every column of the inverse
  for (int k = nb - 1; k >= 0; --k) {
    const double piv = M[(size_t)k * nb + k];
    for (int j = 0; j < nb; ++j) {
      double s = I[(size_t)k * nb + j];
      for (int i = k + 1; i < nb; ++i) s -= M[(size_t)k * nb + i] * I[(size_t)i * nb + j];
      I[(size_t)k * nb + j] = s / piv;
    }
  }
  out.resize((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) out[(size_t)i * n + j] = I[(size_t)i * nb + j];
  return STOKES_OK;
}

}  // namespace

// ------------------------------------------------------------- ledger
namespace {

inline size_t esz(const stokes_handle* h) { return h->prec == STOKES_FP32 ? 4 : 8; }

template <typename T>
const T* kval(const DevCSR& A);
template <>
const float* kval<float>(const DevCSR& A) { return A.v32; }
template <>
const double* kval<double>(const DevCSR& A) { return A.v64; }

// bytes of one SpMV: values + columns + row pointers + x gathered once per
// column + b read (residual modes) + y written (read too when adding)
double spmv_bytes(const DevCSR& A, size_t sv, size_t sx, size_t sb, size_t sy, int mode) {
  double b = double(A.nnz) * (sv + 4) + 4.0 * (A.nrows + 1) + double(A.ncols) * sx + double(A.nrows) * sy;
  if (mode == SPMV_RES || mode == SPMV_SCALED_RES) b += double(A.nrows) * sb;
  if (mode == SPMV_ADD) b += double(A.nrows) * sy;
  if (mode == SPMV_SCALED_RES) b += double(A.nrows);  // row kinds
  return b;
}

template <typename TA, typename TX, typename TB, typename TY, typename TACC>
int L_spmv(stokes_handle* h, const DevCSR& A, const TA* val, const TX* x, const TB* b, TY* y, int mode,
           double s0 = 0, double s1 = 0, const uint8_t* kind = nullptr) {
  if (h->led.count) {
    h->led.bytes += spmv_bytes(A, sizeof(TA), sizeof(TX), sizeof(TB), sizeof(TY), mode);
    h->led.launches += A.nrows > 0;
    return STOKES_OK;
  }
  CK((spmv<TA, TX, TB, TY, TACC>(A, val, x, b, y, mode, s0, s1, kind, h->st)));
  return STOKES_OK;
}

template <typename T, typename TR>
int L_apply(stokes_handle* h, const Level& lv, const TR* r, T* yp) {
  const DevPatches& p = lv.pat;
  if (h->led.count) {
    // factors + patch index lists + output positions + per-patch metadata + gathered r + output
    h->led.bytes += double(p.fac_elems) * sizeof(T) + double(p.nslots) * (4 + 4 + sizeof(TR) + sizeof(T)) +
                    double(p.npatch) * (4 + 4 + 4 + 8 + 4);
    for (int b = 0; b < kTmaBins; ++b) h->led.launches += p.nsmall > 0 && p.bins[b].count > 0;
    h->led.launches += p.nlarge > 0;
    return STOKES_OK;
  }
  CK((vanka_apply<T, TR>(p, r, yp, h->st, &h->fj)));
  return STOKES_OK;
}

template <typename T>
int L_scatter(stokes_handle* h, const Level& lv, const T* yp, T* x, double omega, int mode,
              const double* r64 = nullptr, double* out64 = nullptr, double* x64 = nullptr, T* xadd = nullptr) {
  const DevPatches& p = lv.pat;
  if (h->led.count) {
    double b = 4.0 * (lv.n + 1) + double(p.nslots) * sizeof(T);
    if (mode == 0) b += double(lv.n) * sizeof(T);
    else if (mode == 1) b += 2.0 * lv.n * sizeof(T);
    else b += double(lv.n) * (sizeof(T) + 1 + 8);
    if (x64 && mode != 2) b += 8.0 * lv.n;
    if (xadd) b += 2.0 * lv.n * sizeof(T);
    h->led.bytes += b;
    h->led.launches += 1;
    return STOKES_OK;
  }
  CK(vanka_scatter<T>(p, lv.n, yp, x, omega, mode, h->dir0, r64, out64, h->st, x64, xadd));
  return STOKES_OK;
}

template <typename TI, typename TO>
int L_cast(stokes_handle* h, int64_t n, const TI* in, TO* out) {
  if (h->led.count) {
    h->led.bytes += double(n) * (sizeof(TI) + sizeof(TO));
    h->led.launches += n > 0;
    return STOKES_OK;
  }
  CK((cast_copy<TI, TO>(n, in, out, h->st)));
  return STOKES_OK;
}

template <typename T, typename TI>
int L_axpy(stokes_handle* h, int64_t n, double a, const TI* x, T* y) {
  if (h->led.count) {
    h->led.bytes += double(n) * (sizeof(TI) + 2 * sizeof(T));
    h->led.launches += n > 0;
    return STOKES_OK;
  }
  CK((axpy_into<T, TI>(n, a, x, y, h->st)));
  return STOKES_OK;
}

template <typename T>
int L_diag_scale(stokes_handle* h, int64_t n, const T* d, const T* u, T* z) {
  if (h->led.count) {
    h->led.bytes += 3.0 * n * sizeof(T);
    h->led.launches += n > 0;
    return STOKES_OK;
  }
  CK(diag_scale<T>(n, d, u, z, h->st));
  return STOKES_OK;
}

template <typename T>
int L_zero(stokes_handle* h, int64_t n, T* y) {
  if (h->led.count) {
    h->led.bytes += double(n) * sizeof(T);
    h->led.launches += n > 0;
    return STOKES_OK;
  }
  CK(fill_zero<T>(n, y, h->st));
  return STOKES_OK;
}

template <typename T>
int L_finalize(stokes_handle* h, int64_t n, const T* x, const double* r64, double* out) {
  if (h->led.count) {
    h->led.bytes += double(n) * (sizeof(T) + 1 + 8);
    h->led.launches += n > 0;
    return STOKES_OK;
  }
  CK(finalize_out<T>(n, x, h->dir0, r64, out, h->st));
  return STOKES_OK;
}

template <typename T>
int L_coarse(stokes_handle* h, const Level& lv, const T* b, T* y) {
  const CoarseSet& c = lv.coarse;
  if (c.nblocks == 0) return STOKES_OK;
  if (h->led.count) {
    h->led.bytes += double(c.kinv_elems) * 8.0 + 2.0 * sizeof(T) * std::sqrt(double(c.kinv_elems));
    h->led.launches += 1;
    return STOKES_OK;
  }
  CK(coarse_solve<T>(c.nblocks, c.boff, c.bn, c.koff, c.Kinv, c.max_n, b, y, h->st));
  return STOKES_OK;
}

template <typename T>
int L_cheb_init(stokes_handle* h, int64_t n, const T* b, const T* dinv, const uint8_t* mask, uint8_t want, double s,
                double theta, T* r, T* d, T* x) {
  if (h->led.count) {
    h->led.bytes += double(n) * (4 * sizeof(T) + (dinv ? sizeof(T) : 0) + (mask ? 1 : 0));
    h->led.launches += n > 0;
    return STOKES_OK;
  }
  CK(cheb_init<T>(n, b, dinv, mask, want, s, theta, r, d, x, h->st));
  return STOKES_OK;
}

template <typename T>
int L_cheb_step(stokes_handle* h, const DevCSR& M, const T* val, const T* w, const T* dinv, T* x, T* r, const T* din,
                T* dout, double alpha, double beta) {
  if (h->led.count) {
    h->led.bytes += double(M.nnz) * (sizeof(T) + 4) + 4.0 * (M.nrows + 1) + double(M.ncols) * sizeof(T) +
                    double(M.nrows) * sizeof(T) * (6 + (dinv ? 1 : 0));
    h->led.launches += M.nrows > 0;
    return STOKES_OK;
  }
  CK(cheb_step<T>(M, val, w, dinv, x, r, din, dout, alpha, beta, h->st));
  return STOKES_OK;
}

template <typename T>
int L_cheb_first(stokes_handle* h, const DevCSR& M, const T* val, const T* b, double s, double theta, T* x, T* r,
                 T* dout, double alpha, double beta, bool accumulate) {
  if (h->led.count) {
    h->led.bytes += double(M.nnz) * (sizeof(T) + 4) + 4.0 * (M.nrows + 1) + double(M.ncols) * sizeof(T) +
                    double(M.nrows) * sizeof(T) * (accumulate ? 5 : 4);
    h->led.launches += M.nrows > 0;
    return STOKES_OK;
  }
  CK(cheb_first<T>(M, val, b, s, theta, x, r, dout, alpha, beta, accumulate, h->st));
  return STOKES_OK;
}

template <typename T>
int L_restrict_res(stokes_handle* h, const Level& L, const T* b, const T* x, T* y) {
  if (h->led.count) {
    h->led.bytes += double(L.R.nnz + L.RK.nnz) * (sizeof(T) + 4) + 8.0 * (L.R.nrows + 1) +
                    double(L.R.ncols + L.RK.ncols + L.R.nrows) * sizeof(T);
    h->led.launches += L.R.nrows > 0;
    return STOKES_OK;
  }
  CK(restrict_res<T>(L.R, kval<T>(L.R), b, L.RK, kval<T>(L.RK), x, y, h->st));
  return STOKES_OK;
}

template <typename TI, typename TO>
int L_scatter_rows(stokes_handle* h, int64_t n, const TI* in, const int* rows, TO* out) {
  if (h->led.count) {
    h->led.bytes += double(n) * (sizeof(TI) + 4 + sizeof(TO));
    h->led.launches += n > 0;
    return STOKES_OK;
  }
  CK((scatter_rows<TI, TO>(n, in, rows, out, h->st)));
  return STOKES_OK;
}

// Chebyshev semi-iteration from a zero guess for rhs (masked rows, scaled by
// s) on the interval [lo, hi]: x ~= M^-1 rhs.  For the Schur operator
// B B^T (isS) every step applies B^T into tS and then B.
template <typename T>
int cheb_run(stokes_handle* h, const DevCSR& M, const T* mval, const DevCSR* BT, const T* btval, T* tS,
             const T* dinv, const T* rhs, const uint8_t* mask, uint8_t want, double s, double lo, double hi,
             int degree, T* x, T* r, T* d0, T* d1, int64_t n, bool accumulate = false) {
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  double rho = 1.0 / sigma;
  T* dc = d0;
  T* dn = d1;
  int k = 0;
  if (!BT && !dinv && !mask && degree > 0 && M.nrows == n) {
    // initialisation fused into the first step (x accumulates with `accumulate`)
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    TRY(L_cheb_first<T>(h, M, mval, rhs, s, theta, x, r, dn, rho_new * rho, 2.0 * rho_new / delta, accumulate));
    std::swap(dc, dn);
    rho = rho_new;
    k = 1;
  } else {
    if (accumulate) return fail(STOKES_ERR_INVALID_ARG, "internal: accumulating Chebyshev needs the fused first step");
    TRY(L_cheb_init<T>(h, n, rhs, dinv, mask, want, s, theta, r, d0, x));
  }
  for (; k < degree; ++k) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    const double alpha = rho_new * rho, beta = 2.0 * rho_new / delta;
    const T* w = dc;
    if (BT) {
      TRY((L_spmv<T, T, T, T, T>(h, *BT, btval, dc, (const T*)nullptr, tS, SPMV_SET)));
      w = tS;
    }
    TRY(L_cheb_step<T>(h, M, mval, w, dinv, x, r, dc, dn, alpha, beta));
    std::swap(dc, dn);
    rho = rho_new;
  }
  return STOKES_OK;
}

}  // namespace

namespace {
int check_pipeline_errors(stokes_handle* h);
}

// ------------------------------------------------------------- the cycle
namespace {

// One DLSC sweep (Alg. 2) on level l: momentum, continuity and
// pressure-correction Chebyshev solves, then the velocity correction (D.BT
// already carries Mu^-1, so B D.BT = B Mu^-1 B^T and D.BT q = Mu^-1 B^T q).
template <typename T>
int dlsc_sweep_split(stokes_handle* h, std::vector<Level>& lvs, int l, T* x, const T* b);

template <typename T>
int dlsc_sweep(stokes_handle* h, std::vector<Level>& lvs, int l, T* x, const T* b) {
  Level& L = lvs[l];
  DLSCData& D = L.dl;
  if (D.p0 > 0) return dlsc_sweep_split<T>(h, lvs, l, x, b);
  T** v = reinterpret_cast<T**>(D.v);
  T *res = v[0], *vs = v[1], *q = v[2], *dp = v[3], *t1 = v[4], *t2 = v[5], *cr = v[6], *c0 = v[7], *c1 = v[8];
  const int64_t n = L.n;
  const double fa = std::pow(0.5, h->dim);
  // res = [f - A u - B^T p; g - B u]
  TRY((L_spmv<T, T, T, T, T>(h, L.K, kval<T>(L.K), x, b, res, SPMV_RES)));
  // v* ~ A^-1 (f - A u - B^T p)
  TRY(cheb_run<T>(h, D.A, kval<T>(D.A), nullptr, nullptr, nullptr, nullptr, res, D.kind, 0, 1.0, fa * D.lamA,
                  1.1 * D.lamA, h->cheb_deg[0], vs, cr, c0, c1, n));
  // q ~ S^-1 (g - B (u + v*)),  S = B Mu^-1 B^T
  TRY((L_spmv<T, T, T, T, T>(h, D.B, kval<T>(D.B), vs, res, t1, SPMV_RES)));
  TRY(cheb_run<T>(h, D.B, kval<T>(D.B), &D.BT, kval<T>(D.BT), t2, nullptr, t1, D.kind, 1, 1.0, fa * D.lamS,
                  1.1 * D.lamS, h->cheb_deg[1], q, cr, c0, c1, n));
  // dp ~ S^-1 ( -(B Mu^-1 A Mu^-1 B^T) q )
  TRY((L_spmv<T, T, T, T, T>(h, D.BT, kval<T>(D.BT), q, (const T*)nullptr, t1, SPMV_SET)));
  TRY((L_spmv<T, T, T, T, T>(h, D.A, kval<T>(D.A), t1, (const T*)nullptr, t2, SPMV_SET)));
  T* ta = t2;  // A Mu^-1 B^T q
  T* tb = t1;
  if (D.muinv) {
    TRY(L_diag_scale<T>(h, n, reinterpret_cast<const T*>(D.muinv), t2, t1));
    std::swap(ta, tb);
  }
  TRY((L_spmv<T, T, T, T, T>(h, D.B, kval<T>(D.B), ta, (const T*)nullptr, tb, SPMV_SET)));
  TRY(cheb_run<T>(h, D.B, kval<T>(D.B), &D.BT, kval<T>(D.BT), ta, nullptr, tb, D.kind, 1, -1.0, fa * D.lamS,
                  1.1 * D.lamS, h->cheb_deg[2], dp, cr, c0, c1, n));
  // u += v* + Mu^-1 B^T q ;  p += dp
  TRY((L_axpy<T, T>(h, n, 1.0, vs, x)));
  TRY((L_axpy<T, T>(h, n, 1.0, dp, x)));
  TRY((L_spmv<T, T, T, T, T>(h, D.BT, kval<T>(D.BT), q, (const T*)nullptr, x, SPMV_ADD)));
  return STOKES_OK;
}

// The same sweep on a level whose velocity rows [0, p0) precede its
// pressure rows [p0, n): every step runs on its own row range (the momentum
// solve and B^T on the velocity rows, B and the Schur solves on the pressure
// rows, whose vectors are the level vectors from p0 on), so no launch spends
// threads or bandwidth on rows the block leaves empty; each Schur Chebyshev
// step is one launch on the assembled S = B Mu^-1 B^T instead of B^T then B,
// and the pressure-correction right-hand side one SpMV with the assembled
// T = B Mu^-1 A Mu^-1 B^T instead of four launches.
template <typename T>
int dlsc_sweep_split(stokes_handle* h, std::vector<Level>& lvs, int l, T* x, const T* b) {
  Level& L = lvs[l];
  DLSCData& D = L.dl;
  T** v = reinterpret_cast<T**>(D.v);
  T *res = v[0], *vs = v[1], *q = v[2], *dp = v[3], *t1 = v[4], *cr = v[6], *c0 = v[7], *c1 = v[8];
  const int64_t nv = D.p0, np = L.n - D.p0;
  auto P = [nv](T* p) { return p + nv; };
  const double fa = std::pow(0.5, h->dim);
  // without a pressure-pressure block the momentum and pressure corrections
  // accumulate into x directly, and g - B (u + v*) is the pressure residual
  // of the updated x
  const bool acc = D.pp_zero;
  // res = [f - A u - B^T p; g - B u]
  TRY((L_spmv<T, T, T, T, T>(h, L.K, kval<T>(L.K), x, b, res, SPMV_RES)));
  // v* ~ A^-1 (f - A u - B^T p)
  TRY(cheb_run<T>(h, D.A, kval<T>(D.A), nullptr, nullptr, nullptr, nullptr, res, nullptr, 0, 1.0, fa * D.lamA,
                  1.1 * D.lamA, h->cheb_deg[0], acc ? x : vs, cr, c0, c1, nv, acc));
  // q ~ S^-1 (g - B (u + v*)),  S = B Mu^-1 B^T
  if (acc)
    TRY((L_spmv<T, T, T, T, T>(h, D.B, kval<T>(D.B), x, P(const_cast<T*>(b)), P(t1), SPMV_RES)));
  else
    TRY((L_spmv<T, T, T, T, T>(h, D.B, kval<T>(D.B), vs, P(res), P(t1), SPMV_RES)));
  TRY(cheb_run<T>(h, D.S, kval<T>(D.S), nullptr, nullptr, nullptr, nullptr, P(t1), nullptr, 1, 1.0, fa * D.lamS,
                  1.1 * D.lamS, h->cheb_deg[1], P(q), P(cr), P(c0), P(c1), np));
  // dp ~ S^-1 ( -(B Mu^-1 A Mu^-1 B^T) q ), the right-hand side by the assembled T
  TRY((L_spmv<T, T, T, T, T>(h, D.T, kval<T>(D.T), P(q), (const T*)nullptr, P(t1), SPMV_SET)));
  TRY(cheb_run<T>(h, D.S, kval<T>(D.S), nullptr, nullptr, nullptr, nullptr, P(t1), nullptr, 1, -1.0, fa * D.lamS,
                  1.1 * D.lamS, h->cheb_deg[2], acc ? P(x) : P(dp), P(cr), P(c0), P(c1), np, acc));
  // u += v* + Mu^-1 B^T q ;  p += dp
  if (!acc) {
    TRY((L_axpy<T, T>(h, nv, 1.0, vs, x)));
    TRY((L_axpy<T, T>(h, np, 1.0, P(dp), P(x))));
  }
  TRY((L_spmv<T, T, T, T, T>(h, D.BT, kval<T>(D.BT), P(q), (const T*)nullptr, x, SPMV_ADD)));
  return STOKES_OK;
}

// Krylov-wrapped relaxation (Sec. 3.3.1): k steps of flexible GMRES on
// K e = b - K x from e = 0, right-preconditioned by one undamped Vanka sweep
// per step (classical Gram-Schmidt on unnormalised vectors, per-instance
// scalars on the device), then x += Z y.  zero_guess: x starts at 0 and
// the residual is b.  On level 0 the update also writes the FP64 copy x64
// and/or the cycle output out64.
template <typename T>
int relax_krylov(stokes_handle* h, std::vector<Level>& lvs, int l, T* x, const T* b, int k, bool zero_guess,
                 const double* r64, double* out64, double* x64) {
  Level& L = lvs[l];
  const int64_t n = L.n;
  T* U = reinterpret_cast<T*>(L.kV);
  T* Z = reinterpret_cast<T*>(L.kZ);
  T* yp = reinterpret_cast<T*>(L.yp);
  const int lds = L.lds;
  const KrChunks& ch = L.kch;
  const double Tb = sizeof(T);
  const T* r = b;
  if (!zero_guess) {
    TRY((L_spmv<T, T, T, T, T>(h, L.K, kval<T>(L.K), x, b, U, SPMV_RES)));
    r = U;
  }
  if (h->led.count) {
    // ||r||^2 (+ copy); per step: projections and the orthogonalised update + norm; x update
    double bytes = (zero_guess ? 2.0 : 1.0) * n * Tb;
    for (int j = 0; j < k; ++j) bytes += (j + 2) * n * Tb + (j + 3) * n * Tb;
    bytes += (k + (zero_guess ? 1 : 2)) * n * Tb + (x64 ? 8.0 * n : 0.0) + (out64 ? 17.0 * n : 0.0);
    h->led.bytes += bytes;
    h->led.launches += 1 + 2 * k + 1;
  } else {
    CK(kr_norm0<T>(ch, r, U, L.kpart, L.ldp, L.kcnt, L.kS, lds, h->st));
  }
  for (int j = 0; j < k; ++j) {
    T* uj = U + (size_t)j * n;
    T* zj = Z + (size_t)j * n;
    T* w = U + (size_t)(j + 1) * n;
    if (L.jacobi) {
      TRY(L_diag_scale<T>(h, L.n, reinterpret_cast<const T*>(L.dinv), uj, zj));
    } else {
      TRY((L_apply<T, T>(h, L, uj, yp)));
      TRY(L_scatter<T>(h, L, yp, zj, 1.0, 0));
    }
    TRY((L_spmv<T, T, T, T, T>(h, L.K, kval<T>(L.K), zj, (const T*)nullptr, w, SPMV_SET)));
    if (h->led.count) continue;
    CK(kr_project<T>(ch, j, k, U, n, w, L.kpart, L.ldp, L.kcnt, L.kS, lds, h->st));
    CK(kr_orthogonalise<T>(ch, j, k, U, n, w, L.kpart, L.ldp, L.kcnt, L.kS, lds, h->st));
  }
  if (!h->led.count)
    CK(kr_update<T>(ch, k, Z, n, L.kS, lds, x, zero_guess ? 1 : 0, x64, h->dir0, r64, out64, h->st));
  return STOKES_OK;
}

// nsweeps sweeps of x <- x + omega M^-1 (b - K x) (Eq. vanka); the first
// sweep from a zero guess needs no residual (r = b).  When out64 is given,
// the last scatter writes the level-0 output (Dirichlet rows take r64).
// A DLSC level runs nsweeps calls of dlsc_sweeps DLSC sweeps instead.
template <typename T>
int relax(stokes_handle* h, std::vector<Level>& lvs, int l, T* x, const T* b, int nsweeps, bool zero_guess,
          const double* r64 = nullptr, double* out64 = nullptr, double* x64 = nullptr, T* xadd = nullptr) {
  Level& L = lvs[l];
  if (xadd && (L.krylov || L.dlsc || L.jacobi || nsweeps < 1 || out64))
    return fail(STOKES_ERR_INVALID_ARG, "internal: accumulate target on a non-Vanka relaxation");
  if (L.krylov) {
    if (nsweeps == 0) {
      if (zero_guess) TRY(L_zero<T>(h, L.n, x));
      if (out64) TRY(L_finalize<T>(h, L.n, x, r64, out64));
      else if (x64) TRY((L_cast<T, double>(h, L.n, x, x64)));
      return STOKES_OK;
    }
    return relax_krylov<T>(h, lvs, l, x, b, nsweeps, zero_guess, r64, out64, x64);
  }
  if (L.dlsc) {
    if (zero_guess) TRY(L_zero<T>(h, L.n, x));
    for (int s = 0; s < nsweeps * h->dlsc_sweeps; ++s) TRY(dlsc_sweep<T>(h, lvs, l, x, b));
    // level 0: the cycle output (Dirichlet rows take r) or the FP64 copy of x
    if (out64) TRY(L_finalize<T>(h, L.n, x, r64, out64));
    else if (x64) TRY((L_cast<T, double>(h, L.n, x, x64)));
    return STOKES_OK;
  }
  T* r = reinterpret_cast<T*>(L.r);
  T* yp = reinterpret_cast<T*>(L.yp);
  if (nsweeps == 0 && zero_guess) TRY(L_zero<T>(h, L.n, x));
  for (int s = 0; s < nsweeps; ++s) {
    const bool last_out = out64 && s == nsweeps - 1;
    double* xd = s == nsweeps - 1 ? x64 : nullptr;
    T* xa = s == nsweeps - 1 ? xadd : nullptr;
    if (s == 0 && zero_guess) {
      TRY((L_apply<T, T>(h, L, b, yp)));
      TRY(L_scatter<T>(h, L, yp, x, L.omega, last_out ? 2 : 0, r64, out64, xd, xa));
    } else {
      TRY((L_spmv<T, T, T, T, T>(h, L.K, kval<T>(L.K), x, b, r, SPMV_RES)));
      TRY((L_apply<T, T>(h, L, r, yp)));
      TRY(L_scatter<T>(h, L, yp, x, L.omega, last_out ? 2 : 1, r64, out64, xd, xa));
    }
  }
  return STOKES_OK;
}

// Galerkin V-cycle on level l of the hierarchy lvs (Eq. TG-operator for
// the DC cycle's K1 hierarchy, l >= 1; the SA cycles of BTP from l = 0),
// zero initial guess: input lvs[l].b, output lvs[l].x.  Instances whose
// coarsest level is l take the exact (bordered) solve on their segment.
template <typename T>
int vcycle(stokes_handle* h, std::vector<Level>& lvs, int l) {
  Level& L = lvs[l];
  T* x = reinterpret_cast<T*>(L.x);
  T* b = reinterpret_cast<T*>(L.b);
  if (l == (int)lvs.size() - 1) return L_coarse<T>(h, L, b, x);
  const bool main = &lvs == &h->lv;
  const bool relax_here = (L.has_patches || L.dlsc || L.jacobi) && !(main && h->schedule == STOKES_DC_SKIP1 && l == 1);
  const int nu1 = main ? h->nu1 : h->btp_steps, nu2 = main ? h->nu2 : h->btp_steps;
  if (relax_here) TRY(relax<T>(h, lvs, l, x, b, nu1, true));
  else TRY(L_zero<T>(h, L.n, x));
  TRY(L_coarse<T>(h, L, b, x));
  T* r = reinterpret_cast<T*>(L.r);
  Level& C = lvs[l + 1];
  if (main && L.hasRK) {
    TRY(L_restrict_res<T>(h, L, b, x, reinterpret_cast<T*>(C.b)));
  } else {
    TRY((L_spmv<T, T, T, T, T>(h, L.K, kval<T>(L.K), x, b, r, SPMV_RES)));
    TRY((L_spmv<T, T, T, T, T>(h, L.R, kval<T>(L.R), r, (const T*)nullptr, reinterpret_cast<T*>(C.b), SPMV_SET)));
  }
  TRY(vcycle<T>(h, lvs, l + 1));
  TRY((L_spmv<T, T, T, T, T>(h, L.P, kval<T>(L.P), reinterpret_cast<const T*>(C.x), (const T*)nullptr, x, SPMV_ADD)));
  // level 1 of the DC cycle with P0 = I: the last scatter of the
  // post-relaxation also adds x1 to x0 (dc_cycle then skips x0 += x1)
  T* fold = main && l == 1 && h->fold_x0 && relax_here && nu2 > 0 && !L.krylov && !L.dlsc && !L.jacobi
                ? reinterpret_cast<T*>(h->fold_x0)
                : nullptr;
  if (relax_here) TRY(relax<T>(h, lvs, l, x, b, nu2, false, nullptr, nullptr, nullptr, fold));
  if (fold) h->folded = true;
  return STOKES_OK;
}

// Scott-Vogelius: d = eta (r - K0 x) in FP64; level-1 right-hand side =
// velocity injection of d, pressure = Mcg^-1 Pi^T M_dg d_p by mcg_deg
// Chebyshev-Jacobi steps on the interval [mcg_lo, mcg_hi] (FP64).
template <typename T>
int restrict0_sv_t(stokes_handle* h, const double* x0, const double* r64) {
  Level& L0 = h->lv[0];
  Level& L1 = h->lv[1];
  T* b1 = reinterpret_cast<T*>(L1.b);
  TRY((L_spmv<double, double, double, double, double>(h, L0.K, L0.K.v64, x0, r64, h->d0buf, SPMV_SCALED_RES,
                                                      h->eta_u, h->eta_p, h->kind0)));
  TRY((L_spmv<double, double, double, T, double>(h, h->R0v, h->R0v.v64, h->d0buf, (const double*)nullptr, b1,
                                                 SPMV_SET)));
  TRY((L_spmv<double, double, double, double, double>(h, h->R0q, h->R0q.v64, h->d0buf, (const double*)nullptr,
                                                      h->cv[0], SPMV_SET)));
  TRY(cheb_run<double>(h, h->Mcg, h->Mcg.v64, nullptr, nullptr, nullptr, h->mdinv, h->cv[0], nullptr, 0, 1.0,
                       h->mcg_lo, h->mcg_hi, h->mcg_deg, h->cv[1], h->cv[2], h->cv[3], h->cv[4], h->ncg));
  TRY((L_scatter_rows<double, T>(h, h->ncg, h->cv[1], h->prow1, b1)));
  return STOKES_OK;
}

int restrict0_sv(stokes_handle* h, const double* x0, const double* r64) {
  return h->prec == STOKES_FP32 ? restrict0_sv_t<float>(h, x0, r64) : restrict0_sv_t<double>(h, x0, r64);
}

// z = M_dc^-1 r (Eq. TG-operator-full, gamma = 1), zero initial guess.
template <typename T>
int dc_cycle(stokes_handle* h, const double* r64, double* z64) {
  Level& L0 = h->lv[0];
  Level& L1 = h->lv[1];
  T* x0 = reinterpret_cast<T*>(L0.x);
  const T* r0;
  if (sizeof(T) == 8) {
    r0 = reinterpret_cast<const T*>(r64);
  } else {
    // inside FGMRES the kernel that forms r64 also wrote its FP32 copy
    if (!h->r32_ready) TRY((L_cast<double, T>(h, L0.n, r64, reinterpret_cast<T*>(L0.b))));
    r0 = reinterpret_cast<const T*>(L0.b);
  }
  const bool skip0 = h->schedule == STOKES_DC_SKIP0 || !(L0.has_patches || L0.dlsc);
  // an FP32 cycle also keeps x in FP64 for the FP64 residual of the DC step,
  // so that residual converts each entry once instead of once per nonzero
  double* x0d = sizeof(T) == 8 ? reinterpret_cast<double*>(x0) : h->x0_64;
  const bool pre = !skip0 && h->nu1 > 0;
  if (pre) TRY(relax<T>(h, h->lv, 0, x0, r0, h->nu1, true, nullptr, nullptr, sizeof(T) == 8 ? nullptr : x0d));
  else {
    TRY(L_zero<T>(h, L0.n, x0));
    if (sizeof(T) != 8) TRY(L_zero<double>(h, L0.n, x0d));
  }
  // DC residual in FP64: d = eta (r - K0 x), then R0 (Eq. interp)
  if (h->disc == STOKES_TH && L0.Pident) {  // R0 = injection, fused into the residual
    TRY((L_spmv<double, double, double, T, double>(h, L0.K, L0.K.v64, x0d, r64, reinterpret_cast<T*>(L1.b),
                                                   SPMV_SCALED_RES, h->eta_u, h->eta_p, h->kind0)));
  } else if (h->disc == STOKES_TH) {  // a general R0 = P0^T (HO-AMG hierarchies)
    TRY((L_spmv<double, double, double, double, double>(h, L0.K, L0.K.v64, x0d, r64, h->d0buf, SPMV_SCALED_RES,
                                                        h->eta_u, h->eta_p, h->kind0)));
    TRY((L_spmv<double, double, double, T, double>(h, L0.R, L0.R.v64, h->d0buf, (const double*)nullptr,
                                                   reinterpret_cast<T*>(L1.b), SPMV_SET)));
  } else {
    TRY(restrict0_sv(h, x0d, r64));
  }
  h->fold_x0 = L0.Pident ? x0 : nullptr;
  h->folded = false;
  const int rc1 = vcycle<T>(h, h->lv, 1);
  h->fold_x0 = nullptr;
  TRY(rc1);
  if (L0.Pident) {  // P0 = I
    if (!h->folded) TRY((L_axpy<T, T>(h, L0.n, 1.0, reinterpret_cast<const T*>(L1.x), x0)));
  }
  else TRY((L_spmv<T, T, T, T, T>(h, L0.P, kval<T>(L0.P), reinterpret_cast<const T*>(L1.x), (const T*)nullptr, x0, SPMV_ADD)));
  if (!skip0 && h->nu2 > 0) TRY(relax<T>(h, h->lv, 0, x0, r0, h->nu2, false, r64, z64));
  else TRY(L_finalize<T>(h, L0.n, x0, r64, z64));
  return STOKES_OK;
}

template <typename T>
int L_btp_out(stokes_handle* h, int64_t nu, int64_t np, const T* du, const T* dp, double sp, const double* r64,
              double* z) {
  if (h->led.count) {
    h->led.bytes += double(nu) * (sizeof(T) + 1 + 8 + 8) + double(np) * (sizeof(T) + 8);
    h->led.launches += nu + np > 0;
    return STOKES_OK;
  }
  CK(btp_out<T>(nu, np, du, dp, sp, h->dir0, r64, z, h->st));
  return STOKES_OK;
}

// BTP (Sec. 4): du = Q_A^-1 r_u (SA V-cycle on A), y = r_p - B du,
// Q_B^-1 y (SA V-cycle on M_p / nu, or the exact block inverse), and the
// pressure update dp = -Q_B^-1 y = Q_B^-1 (B du - r_p).
template <typename T>
int btp_cycle(stokes_handle* h, const double* r64, double* z64) {
  Level& A0 = h->btpA[0];
  const int64_t nu = A0.n, np = h->lv[0].n - nu;
  T* tp = reinterpret_cast<T*>(h->btp_tp);
  TRY((L_cast<double, T>(h, nu, r64, reinterpret_cast<T*>(A0.b))));
  TRY((L_cast<double, T>(h, np, r64 + nu, tp)));
  TRY(vcycle<T>(h, h->btpA, 0));
  const T* du = reinterpret_cast<const T*>(A0.x);
  const T* dq;
  if (!h->btpM.empty()) {
    Level& M0 = h->btpM[0];
    TRY((L_spmv<T, T, T, T, T>(h, h->btpB, kval<T>(h->btpB), du, tp, reinterpret_cast<T*>(M0.b), SPMV_RES)));
    TRY(vcycle<T>(h, h->btpM, 0));
    dq = reinterpret_cast<const T*>(M0.x);
  } else {
    T* y = tp + np;
    T* w = tp + 2 * np;
    TRY((L_spmv<T, T, T, T, T>(h, h->btpB, kval<T>(h->btpB), du, tp, y, SPMV_RES)));
    TRY((L_spmv<T, T, T, T, T>(h, h->btpMinv, kval<T>(h->btpMinv), y, (const T*)nullptr, w, SPMV_SET)));
    dq = w;
  }
  return L_btp_out<T>(h, nu, np, du, dq, -1.0, r64, z64);
}

int run_cycle(stokes_handle* h, const double* r, double* z) {
  if (h->precond == STOKES_PRECOND_BTP)
    return h->prec == STOKES_FP32 ? btp_cycle<float>(h, r, z) : btp_cycle<double>(h, r, z);
  return h->prec == STOKES_FP32 ? dc_cycle<float>(h, r, z) : dc_cycle<double>(h, r, z);
}

int cycle_graph(stokes_handle* h, const double* r, double* z, cudaGraphExec_t* out) {
  auto key = std::make_pair((const void*)r, (void*)z);
  auto it = h->graphs.find(key);
  if (it != h->graphs.end()) {
    *out = it->second;
    return STOKES_OK;
  }
  if (h->cycle_launches < 0) {
    h->led = Ledger();
    h->led.count = true;
    int rc0 = run_cycle(h, r, z);
    h->led.count = false;
    TRY(rc0);
    h->cycle_launches = h->led.launches;
  }
  // one plain run first (sets kernel attributes outside capture)
  TRY(run_cycle(h, r, z));
  h->launches += h->cycle_launches;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
  int rc = run_cycle(h, r, z);
  cudaError_t ec = cudaStreamEndCapture(h->st, &g);
  if (rc != STOKES_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  CK(ec);
  cudaGraphExec_t ge = nullptr;
  cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  CK(ei);
  h->graphs[key] = ge;
  *out = ge;
  return STOKES_OK;
}

}  // namespace

// With no caller stream, the handle's own stream is ordered after the work
// already queued on the legacy default stream and before the work queued
// there later, as if the calls ran on the default stream.
namespace {
int join_in(stokes_handle* h) {
  if (!h->own_stream) return STOKES_OK;
  CK(cudaEventRecord(h->ev_in, cudaStreamLegacy));
  CK(cudaStreamWaitEvent(h->st, h->ev_in, 0));
  return STOKES_OK;
}
int join_out(stokes_handle* h) {
  if (!h->own_stream) return STOKES_OK;
  CK(cudaEventRecord(h->ev_out, h->st));
  CK(cudaStreamWaitEvent(cudaStreamLegacy, h->ev_out, 0));
  return STOKES_OK;
}
}  // namespace

// Level data the no-allocation Vanka entry point needs (noalloc.cu).
namespace sd {
int vanka_level_view(stokes_handle* h, int l, VankaView* v) {
  if (!h || l < 0 || l >= h->L) return fail(STOKES_ERR_INVALID_ARG, "level out of range");
  Level& lv = h->lv[l];
  if (!lv.has_patches) return fail(STOKES_ERR_INVALID_ARG, "level has no Vanka patches");
  if (!h->factored) return fail(STOKES_ERR_STATE, "stokes_factor_patches must run first");
  v->pat = &lv.pat;
  v->n = lv.n;
  v->fp32 = h->prec == STOKES_FP32;
  v->st = h->st;
  return STOKES_OK;
}
int stream_join_in(stokes_handle* h) { return join_in(h); }
int stream_join_out(stokes_handle* h) { return join_out(h); }
int set_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace sd

// ------------------------------------------------------------- C ABI
extern "C" {

const char* stokes_last_error(void) { return g_err.c_str(); }

const char* stokes_status_string(int s) {
  switch (s) {
    case STOKES_OK: return "ok";
    case STOKES_NOT_CONVERGED: return "not converged";
    case STOKES_ERR_INVALID_ARG: return "invalid argument";
    case STOKES_ERR_CUDA: return "CUDA error";
    case STOKES_ERR_OOM: return "out of device memory";
    case STOKES_ERR_SINGULAR_PATCH: return "singular patch";
    case STOKES_ERR_NAN: return "non-finite value";
    case STOKES_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

void stokes_destroy(stokes_handle* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : h->iter_graphs) cudaGraphExecDestroy(kv.second);
  for (auto& e : h->ev_iter)
    if (e) cudaEventDestroy(e);
  if (h->hstat) cudaFreeHost(h->hstat);
  for (void* p : h->allocs) cudaFree(p);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  for (int k = 0; k < kForkMax; ++k) {
    if (h->fj.side[k]) cudaStreamDestroy(h->fj.side[k]);
    if (h->fj.join[k]) cudaEventDestroy(h->fj.join[k]);
  }
  if (h->fj.fork) cudaEventDestroy(h->fj.fork);
  if (h->own_stream && h->st) cudaStreamDestroy(h->st);
  delete h;
}

static bool configure_bin(const DevPatches& dp, TmaBin& bn, int b, int tp, int stages,
                          const std::vector<int64_t>& foff, const std::vector<int>& pptr, size_t T, int nsm);

// Autotuner of the bulk-copy Vanka bins: for every level and bin, time the
// bin's apply for patches-per-tile in {tp/2, tp, 2 tp} and a 2- or 3-stage
// ring (CUDA events, after one warm-up launch) and keep the fastest.  The
// per-patch arithmetic does not depend on the tiling, so results are
// unchanged; captured graphs are dropped because they hold the old launch
// configurations.
int stokes_autotune(stokes_handle* h, int32_t reps) {
  if (!h) return fail(STOKES_ERR_INVALID_ARG, "null handle");
  if (!h->factored) return fail(STOKES_ERR_STATE, "stokes_factor_patches must run first");
  if (reps < 1) reps = 5;
  TRY(join_in(h));
  int nsm = 0, dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const size_t T = esz(h);
  const bool f32 = h->prec == STOKES_FP32;
  // every timed launch starts with a cold L2, as inside a cycle (whose
  // working set is far larger than L2): back-to-back launches would find
  // part of the factors still cached and favour the wrong configuration
  if (!h->flush) {
    h->flush_bytes = size_t(256) << 20;
    TRY(dalloc(h, reinterpret_cast<char**>(&h->flush), h->flush_bytes));
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::string rep = "{\"bins\": [";
  bool first = true;
  int rc = STOKES_OK;
  for (int l = 0; l < h->L && rc == STOKES_OK; ++l) {
    Level& lv = h->lv[l];
    if (!lv.has_patches || !lv.pat.use_tma) continue;
    DevPatches& dp = lv.pat;
    CK(cudaMemsetAsync(lv.r, 0, (size_t)lv.n * T, h->st));
    for (int b = 0; b < kTmaBins; ++b) {
      TmaBin& bn = dp.bins[b];
      if (bn.count == 0) continue;
      const TmaBin base = bn;
      const int ppw = vanka_tma_bin_ppw(b);
      TmaBin best = base;
      float best_ms = -1.f;
      for (int tp : {base.tp / 2, base.tp, base.tp * 2}) {
        if (tp < 4 * ppw || tp > 128) continue;
        for (int stages : {2, 3}) {
          TmaBin cand = base;
          if (!configure_bin(dp, cand, b, tp, stages, lv.hfoff, lv.hpptr, T, nsm)) continue;
          bn = cand;
          CK(vanka_apply_bin(dp, b, lv.r, lv.yp, f32, h->st));
          float ms = 0.f;
          for (int q = 0; q < reps; ++q) {
            CK(l2_flush(h->flush, h->flush_bytes, h->st));
            CK(cudaEventRecord(e0, h->st));
            CK(vanka_apply_bin(dp, b, lv.r, lv.yp, f32, h->st));
            CK(cudaEventRecord(e1, h->st));
            CK(cudaEventSynchronize(e1));
            float one = 0.f;
            CK(cudaEventElapsedTime(&one, e0, e1));
            ms += one;
          }
          ms /= reps;
          if (best_ms < 0.f || ms < best_ms) {
            best_ms = ms;
            best = cand;
          }
        }
      }
      bn = best;
      char buf[256];
      snprintf(buf, sizeof buf,
               "%s{\"level\": %d, \"bin\": %d, \"patches\": %d, \"tile_patches\": %d, \"stages\": %d, "
               "\"grid\": %d, \"us\": %.2f}",
               first ? "" : ", ", l, b, bn.count, bn.tp, bn.stages, bn.grid, best_ms * 1000.f);
      rep += buf;
      first = false;
    }
  }
  rep += "]}";
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TRY(check_pipeline_errors(h));
  for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
  for (auto& kv : h->iter_graphs) cudaGraphExecDestroy(kv.second);
  h->iter_graphs.clear();
  h->tune_report = rep;
  TRY(join_out(h));
  return rc;
}

const char* stokes_autotune_report(const stokes_handle* h) { return h ? h->tune_report.c_str() : "{}"; }

int stokes_galerkin(const stokes_csr* K, const stokes_csr* P, void* cuda_stream, stokes_csr* C) {
  if (!K || !P || !C) return fail(STOKES_ERR_INVALID_ARG, "null argument");
  TRY(check_csr(K, "galerkin K"));
  TRY(check_csr(P, "galerkin P"));
  if (K->nrows != K->ncols || P->nrows != K->nrows)
    return fail(STOKES_ERR_INVALID_ARG, "galerkin: K must be square and P must have K's rows");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  std::vector<int> kcol(K->col, K->col + K->nnz), pcol(P->col, P->col + P->nnz);
  int status = 0;
  int64_t* crp = nullptr;
  int* ccol = nullptr;
  double* cval = nullptr;
  int64_t cnnz = 0;
  cudaError_t e = galerkin_rap(K->nrows, K->rowptr, kcol.data(), K->val, P->ncols, P->rowptr, pcol.data(), P->val,
                               st, &status, &crp, &ccol, &cval, &cnnz);
  if (e != cudaSuccess) {
    delete[] crp;
    delete[] ccol;
    delete[] cval;
    return fail(e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA,
                std::string("galerkin: ") + cudaGetErrorString(e));
  }
  if (status) return fail(STOKES_ERR_INVALID_ARG, "galerkin: a row has more than 4096 partial products");
  C->nrows = P->ncols;
  C->ncols = P->ncols;
  C->nnz = cnnz;
  C->rowptr = crp;
  C->col = ccol;
  C->val = cval;
  return STOKES_OK;
}

void stokes_csr_free(stokes_csr* C) {
  if (!C) return;
  delete[] C->rowptr;
  delete[] C->col;
  delete[] C->val;
  C->rowptr = nullptr;
  C->col = nullptr;
  C->val = nullptr;
  C->nnz = 0;
}

// shared tail of the setup entry points: a failed CUDA call, or a filled CSR
static int setup_csr_out(cudaError_t e, const char* what, int32_t nr, int32_t nc, int64_t nnz, int64_t* rp, int* col,
                         double* val, stokes_csr* out) {
  if (e != cudaSuccess) {
    delete[] rp;
    delete[] col;
    delete[] val;
    return fail(e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  }
  out->nrows = nr;
  out->ncols = nc;
  out->nnz = nnz;
  out->rowptr = rp;
  out->col = col;
  out->val = val;
  return STOKES_OK;
}

int stokes_sa_strength(const stokes_csr* A, double theta, void* cuda_stream, stokes_csr* S) {
  if (!A || !S) return fail(STOKES_ERR_INVALID_ARG, "null argument");
  TRY(check_csr(A, "strength A"));
  if (A->nrows != A->ncols || !(theta >= 0.0)) return fail(STOKES_ERR_INVALID_ARG, "strength: A square, theta >= 0");
  std::vector<int> col(A->col, A->col + A->nnz);
  int64_t* rp = nullptr;
  int* c = nullptr;
  double* v = nullptr;
  int64_t nnz = 0;
  cudaError_t e = sa_strength(A->nrows, A->rowptr, col.data(), A->val, theta,
                              reinterpret_cast<cudaStream_t>(cuda_stream), &rp, &c, &v, &nnz);
  return setup_csr_out(e, "strength", A->nrows, A->nrows, nnz, rp, c, v, S);
}

int stokes_sa_tentative(int32_t n, const int32_t* agg, int32_t naggregates, const double* B, void* cuda_stream,
                        stokes_csr* T, double* Bc) {
  if (n < 0 || naggregates < 0 || (n > 0 && (!agg || !B)) || !T || (naggregates > 0 && !Bc))
    return fail(STOKES_ERR_INVALID_ARG, "tentative: bad arguments");
  std::vector<int> present(naggregates, 0);
  for (int i = 0; i < n; ++i) {
    if (agg[i] < -1 || agg[i] >= naggregates) return fail(STOKES_ERR_INVALID_ARG, "tentative: aggregate out of range");
    if (agg[i] >= 0) present[agg[i]] = 1;
  }
  for (int a = 0; a < naggregates; ++a)
    if (!present[a]) return fail(STOKES_ERR_INVALID_ARG, "tentative: empty aggregate");
  int64_t* rp = nullptr;
  int* c = nullptr;
  double* v = nullptr;
  int64_t nnz = 0;
  cudaError_t e = sa_tentative(n, agg, naggregates, B, reinterpret_cast<cudaStream_t>(cuda_stream), &rp, &c, &v, &nnz,
                               Bc);
  return setup_csr_out(e, "tentative", n, naggregates, nnz, rp, c, v, T);
}

int stokes_sa_smooth(const stokes_csr* A, const stokes_csr* T, double omega, void* cuda_stream, stokes_csr* P) {
  if (!A || !T || !P) return fail(STOKES_ERR_INVALID_ARG, "null argument");
  TRY(check_csr(A, "smooth A"));
  TRY(check_csr(T, "smooth T"));
  if (A->nrows != A->ncols || T->nrows != A->nrows)
    return fail(STOKES_ERR_INVALID_ARG, "smooth: A must be square and T must have A's rows");
  std::vector<int> acol(A->col, A->col + A->nnz), tcol(T->col, T->col + T->nnz);
  int status = 0;
  int64_t* rp = nullptr;
  int* c = nullptr;
  double* v = nullptr;
  int64_t nnz = 0;
  cudaError_t e = sa_smooth(A->nrows, A->rowptr, acol.data(), A->val, T->ncols, T->rowptr, tcol.data(), T->val, omega,
                            reinterpret_cast<cudaStream_t>(cuda_stream), &status, &rp, &c, &v, &nnz);
  if (e == cudaSuccess && status) return fail(STOKES_ERR_INVALID_ARG, "smooth: a row has more than 4096 products");
  return setup_csr_out(e, "smooth", A->nrows, T->ncols, nnz, rp, c, v, P);
}

int stokes_vanka_patches(const stokes_csr* K, const int64_t* field_off, int32_t dim, double rel_tol, void* cuda_stream,
                         stokes_patch_lists* out) {
  if (!K || !field_off || !out || (dim != 2 && dim != 3) || !(rel_tol >= 0.0))
    return fail(STOKES_ERR_INVALID_ARG, "vanka_patches: bad arguments");
  TRY(check_csr(K, "vanka_patches K"));
  if (K->nrows != K->ncols || field_off[0] != 0 || field_off[dim + 1] != K->nrows)
    return fail(STOKES_ERR_INVALID_ARG, "vanka_patches: field offsets do not span K");
  for (int c = 0; c <= dim; ++c)
    if (field_off[c + 1] < field_off[c]) return fail(STOKES_ERR_INVALID_ARG, "vanka_patches: offsets decrease");
  for (int c = 1; c < dim; ++c)
    if (field_off[c + 1] - field_off[c] != field_off[1] - field_off[0])
      return fail(STOKES_ERR_INVALID_ARG, "vanka_patches: velocity components of different sizes");
  std::vector<int> col(K->col, K->col + K->nnz);
  int status = 0, np = 0;
  int64_t* ptr = nullptr;
  int *dof = nullptr, *nvel = nullptr, *npres = nullptr;
  cudaError_t e = vanka_patch_lists(K->nrows, K->rowptr, col.data(), K->val, field_off, dim, rel_tol,
                                    reinterpret_cast<cudaStream_t>(cuda_stream), &status, &np, &ptr, &dof, &nvel,
                                    &npres);
  if (e != cudaSuccess || status) {
    delete[] ptr;
    delete[] dof;
    delete[] nvel;
    delete[] npres;
    if (e != cudaSuccess)
      return fail(e == cudaErrorMemoryAllocation ? STOKES_ERR_OOM : STOKES_ERR_CUDA,
                  std::string("vanka_patches: ") + cudaGetErrorString(e));
    return fail(STOKES_ERR_INVALID_ARG, "vanka_patches: a pressure row has more than 4096 velocity entries");
  }
  out->npatch = np;
  out->ptr = ptr;
  out->dof = dof;
  out->nvel = nvel;
  out->npres = npres;
  return STOKES_OK;
}

void stokes_patch_lists_free(stokes_patch_lists* p) {
  if (!p) return;
  delete[] p->ptr;
  delete[] p->dof;
  delete[] p->nvel;
  delete[] p->npres;
  p->ptr = nullptr;
  p->dof = nullptr;
  p->nvel = nullptr;
  p->npres = nullptr;
  p->npatch = 0;
}

int stokes_num_levels(const stokes_handle* h) { return h ? h->L : 0; }
int64_t stokes_kernel_launches(const stokes_handle* h) { return h ? h->launches : 0; }
int64_t stokes_level_size(const stokes_handle* h, int32_t l) {
  return (h && l >= 0 && l < h->L) ? h->lv[l].n : -1;
}

// DLSC level: the A, B and B^T blocks as level-sized CSRs, row kinds, bounds
// and nine work vectors.
static int setup_dlsc(stokes_handle* h, Level& lv, const stokes_problem* const* probs, int ninst, int l, int dim) {
  HostCSR A, B, BT;
  A.nrows = B.nrows = BT.nrows = A.ncols = B.ncols = BT.ncols = (int)lv.n;
  std::vector<uint8_t> kind(lv.n, 2);
  // level 0 (the P2 grid): Mu = diag(Mu_diag); levels >= 1: Mu = I
  const bool mass = l == 0;
  std::vector<double> muinv(mass ? lv.n : 0, 0.0);
  bool has_pp = false;
  for (int k = 0; k < ninst; ++k) {
    const stokes_problem* p = probs[k];
    if (p->nlevels <= l) continue;
    const stokes_csr* K = &p->K[l];
    const int64_t* off = p->field_off + (size_t)l * (dim + 2);
    const int64_t o = lv.seg_off[k];
    const bool relaxes = p->nlevels - 1 > l;
    if (mass && relaxes)
      for (int64_t i = 0; i < off[dim]; ++i) {
        const double m = p->Mu_diag[i];
        if (!(m > 0) || !std::isfinite(m)) return fail(STOKES_ERR_INVALID_ARG, "Mu_diag entries must be positive");
        muinv[o + i] = 1.0 / m;
      }
    for (int i = 0; i < K->nrows; ++i) {
      const bool vel = i < off[dim];
      if (relaxes) kind[o + i] = vel ? 0 : 1;
      for (int64_t e = K->rowptr[i]; relaxes && e < K->rowptr[i + 1]; ++e) {
        const int c = K->col[e];
        const bool cvel = c < off[dim];
        HostCSR& dst = vel ? (cvel ? A : BT) : (cvel ? B : A);
        if (!vel && !cvel) {  // zero block (a nonzero entry here is left out of A, B, B^T)
          if (K->val[e] != 0.0) has_pp = true;
          continue;
        }
        dst.col.push_back((int)(o + c));
        // B^T rows carry Mu^-1 (velocity row i of B^T scaled by 1/Mu_i)
        dst.val.push_back(mass && vel && !cvel ? K->val[e] * muinv[o + i] : K->val[e]);
      }
      A.rowptr.push_back((int)A.col.size());
      B.rowptr.push_back((int)B.col.size());
      BT.rowptr.push_back((int)BT.col.size());
    }
  }
  // one velocity run followed by one pressure run: keep only the nonempty rows
  int64_t p0 = 0;
  while (p0 < lv.n && kind[p0] == 0) ++p0;
  bool split = p0 > 0 && p0 < lv.n;
  for (int64_t i = p0; split && i < lv.n; ++i) split = kind[i] == 1;
  if (split) {
    auto rows = [](const HostCSR& M, int64_t r0, int64_t r1, int ncols, int shift) {
      HostCSR o;
      o.nrows = (int)(r1 - r0);
      o.ncols = ncols;  // rowptr starts as {0}
      for (int64_t i = r0; i < r1; ++i) {
        for (int e = M.rowptr[i]; e < M.rowptr[i + 1]; ++e) {
          o.col.push_back(M.col[e] - shift);
          o.val.push_back(M.val[e]);
        }
        o.rowptr.push_back((int)o.col.size());
      }
      return o;
    };
    const int nv = (int)p0, np = (int)(lv.n - p0);
    const HostCSR Bp = rows(B, p0, lv.n, nv, 0), BTv = rows(BT, 0, p0, np, nv);
    const HostCSR Av = rows(A, 0, p0, nv, 0);
    // S = B (Mu^-1 B^T), the Schur operator of Alg. 2 (B^T already carries
    // Mu^-1), and T = B Mu^-1 A (Mu^-1 B^T), the operator of the right-hand
    // side of the pressure-correction solve, both on the pressure rows
    const HostCSR S = csr_product(Bp, BTv, nullptr);
    const HostCSR T = csr_product(Bp, csr_product(Av, BTv, mass ? muinv.data() : nullptr), nullptr);
    // the DLSC operators take the sliced-ELLPACK copy from 64 k rows on (their
    // Chebyshev steps and SpMVs measured faster there than on row-block tiles)
    constexpr int kDlscSellRows = 65536;
    TRY(upload_csr(h, lv.dl.T, T, kDlscSellRows));
    TRY(upload_csr(h, lv.dl.A, Av, kDlscSellRows));
    TRY(upload_csr(h, lv.dl.B, Bp, kDlscSellRows));
    TRY(upload_csr(h, lv.dl.BT, BTv, kDlscSellRows));
    TRY(upload_csr(h, lv.dl.S, S, kDlscSellRows));
    lv.dl.p0 = p0;
    lv.dl.pp_zero = !has_pp;
  } else {
    TRY(upload_csr(h, lv.dl.A, A));
    TRY(upload_csr(h, lv.dl.B, B));
    TRY(upload_csr(h, lv.dl.BT, BT));
  }
  TRY(upload(h, &lv.dl.kind, kind));
  if (mass) {
    if (h->prec == STOKES_FP32) {
      std::vector<float> m32(muinv.begin(), muinv.end());
      float* d = nullptr;
      TRY(upload(h, &d, m32));
      lv.dl.muinv = d;
    } else {
      double* d = nullptr;
      TRY(upload(h, &d, muinv));
      lv.dl.muinv = d;
    }
  }
  for (int k = 0; k < ninst; ++k)
    if (probs[k]->nlevels - 1 > l) {
      lv.dl.lamA = probs[k]->lambda_A[l];
      lv.dl.lamS = probs[k]->lambda_S[l];
      break;
    }
  if (!(lv.dl.lamA > 0 && lv.dl.lamS > 0)) return fail(STOKES_ERR_INVALID_ARG, "DLSC eigenvalue bounds must be positive");
  for (int q = 0; q < 9; ++q) {
    char* p = nullptr;
    TRY(dalloc(h, &p, (size_t)lv.n * esz(h)));
    lv.dl.v[q] = p;
  }
  lv.dlsc = true;
  return STOKES_OK;
}

// Scott-Vogelius restriction data: velocity injection R0v (level 1 x level
// 0), the projection right-hand side R0q = Pi^T M_dg and Mcg on the
// compressed pressure rows, the level-1 row of each, 1/diag(Mcg).
static int setup_sv(stokes_handle* h, const stokes_problem* const* probs, int ninst, int dim) {
  Level& L0 = h->lv[0];
  Level& L1 = h->lv[1];
  HostCSR R0v, R0q, Mc;
  R0v.nrows = (int)L1.n;
  R0v.ncols = (int)L0.n;
  std::vector<int> prow;
  std::vector<double> dinv;
  int64_t ncg = 0;
  for (int k = 0; k < ninst; ++k) ncg += probs[k]->Mcg->nrows;
  R0q.nrows = Mc.nrows = Mc.ncols = (int)ncg;
  R0q.ncols = (int)L0.n;
  int64_t cg0 = 0;
  for (int k = 0; k < ninst; ++k) {
    const stokes_problem* p = probs[k];
    const int64_t* o0 = p->field_off;
    const int64_t* o1 = p->field_off + (dim + 2);
    const int64_t s0 = L0.seg_off[k], s1 = L1.seg_off[k];
    for (int64_t i = 0; i < o1[dim + 1]; ++i) {
      if (i < o1[dim]) {
        R0v.col.push_back((int)(s0 + i));
        R0v.val.push_back(1.0);
      }
      R0v.rowptr.push_back((int)R0v.col.size());
    }
    append_block(R0q, p->R0p, s0 + o0[dim]);
    append_block(Mc, p->Mcg, cg0);
    for (int i = 0; i < p->Mcg->nrows; ++i) {
      prow.push_back((int)(s1 + o1[dim] + i));
      double dg = 0.0;
      for (int64_t e = p->Mcg->rowptr[i]; e < p->Mcg->rowptr[i + 1]; ++e)
        if (p->Mcg->col[e] == i) dg = p->Mcg->val[e];
      if (!(dg > 0)) return fail(STOKES_ERR_INVALID_ARG, "Mcg needs a positive diagonal");
      dinv.push_back(1.0 / dg);
    }
    cg0 += p->Mcg->nrows;
  }
  TRY(upload_csr(h, h->R0v, R0v));
  TRY(upload_csr(h, h->R0q, R0q));
  TRY(upload_csr(h, h->Mcg, Mc));
  TRY(upload(h, &h->prow1, prow));
  TRY(upload(h, &h->mdinv, dinv));
  for (int q = 0; q < 5; ++q) TRY(dalloc(h, &h->cv[q], (size_t)ncg));
  TRY(dalloc(h, &h->d0buf, (size_t)L0.n));
  h->ncg = ncg;
  h->mcg_lo = probs[0]->mcg_lo;
  h->mcg_hi = probs[0]->mcg_hi;
  return STOKES_OK;
}

// Krylov-wrapped relaxation on level l: chunk tables over the level's
// instance segments (2048 rows, never straddling an instance), the basis
// vectors and the per-instance scalars.
static int setup_krylov_relax(stokes_handle* h, Level& lv, const stokes_problem* const* probs, int ninst, int l) {
  lv.krylov = true;
  lv.kmax = std::max(std::max(h->nu1, h->nu2), 1);
  const int k = lv.kmax;
  lv.lds = 1 + k * (k + 1) + k;
  lv.ldp = kKrMaxSteps;
  std::vector<int64_t> cb, ce;
  std::vector<int> cs, sb(ninst, 0), se(ninst, 0);
  const int64_t CH = 2048;  // few chunks: each reduction's completion sums one partial per chunk
  for (int q = 0; q < ninst; ++q) {
    sb[q] = (int)cb.size();
    if (lv.seg_off[q] >= 0) {
      const int64_t o = lv.seg_off[q], n = probs[q]->K[l].nrows;
      for (int64_t r = 0; r < n; r += CH) {
        cb.push_back(o + r);
        ce.push_back(o + std::min(n, r + CH));
        cs.push_back(q);
      }
    }
    se[q] = (int)cb.size();
  }
  lv.kch.n = (int)cb.size();
  TRY(upload(h, &lv.kch.beg, cb));
  TRY(upload(h, &lv.kch.end, ce));
  TRY(upload(h, &lv.kch.seg, cs));
  TRY(upload(h, &lv.kch.sbeg, sb));
  TRY(upload(h, &lv.kch.send, se));
  const size_t T = esz(h);
  char *V, *Z;
  TRY(dalloc(h, &V, (size_t)(k + 1) * lv.n * T));
  TRY(dalloc(h, &Z, (size_t)k * lv.n * T));
  lv.kV = V;
  lv.kZ = Z;
  TRY(dalloc(h, &lv.kS, (size_t)ninst * lv.lds));
  TRY(dalloc(h, &lv.kpart, (size_t)std::max(lv.kch.n, 1) * lv.ldp));
  TRY(dalloc(h, &lv.kcnt, (size_t)ninst));
  CK(cudaMemset(lv.kcnt, 0, sizeof(int) * ninst));
  return STOKES_OK;
}

// Tile configuration of a bulk-copy bin for `tp` patches per tile: the
// largest tile's factor, index-list and right-hand-side sizes, the ring
// depth and the persistent grid (CTAs per SM from the occupancy query).
// Returns false when no CTA fits on an SM.
static bool configure_bin(const DevPatches& dp, TmaBin& bn, int b, int tp, int stages,
                          const std::vector<int64_t>& foff, const std::vector<int>& pptr, size_t T, int nsm) {
  bn.tp = tp;
  bn.ntiles = (bn.count + tp - 1) / tp;
  int64_t fb = 0, db = 0, rh = 0;
  for (int t = 0; t < bn.ntiles; ++t) {
    const int i0 = bn.start + t * tp, i1 = std::min(i0 + tp, bn.start + bn.count);
    fb = std::max(fb, (foff[i1] - foff[i0]) * (int64_t)T);
    db = std::max<int64_t>(db, (int64_t)(((pptr[i1] + 3) & ~3) - (pptr[i0] & ~3)) * 4);
    const int cnt = i1 - i0, per = (cnt + 3) / 4;
    for (int w = 0; w < 4; ++w) {
      const int j0 = std::min(i0 + w * per, i1), j1 = std::min(j0 + per, i1);
      rh = std::max<int64_t>(rh, pptr[j1] - pptr[j0]);
    }
  }
  bn.fac_bytes = (int)fb;
  bn.dof_bytes = (int)db;
  bn.rhs_elems = (int)((rh + 3) / 4 * 4);
  bn.stages = stages;
  if (vanka_tma_smem(dp, bn, T) > 220 * 1024) return false;
  const int nb = vanka_tma_blocks_per_sm(dp, bn, b, T);
  if (nb < 1) return false;
  bn.grid = std::min(bn.ntiles, nsm * nb);
  return true;
}

// BTP (Sec. 4): the SA hierarchies of A and of M_p / nu (or the exact
// block inverse), B, Jacobi diagonals, Krylov-relaxation chunks and work
// vectors.  Single-instance handles only.
static int setup_btp_levels(stokes_handle* h, std::vector<Level>& lvs, const stokes_csr* K, const stokes_csr* P,
                            int nl, const char* what) {
  lvs.assign(nl, Level());
  const size_t T = esz(h);
  for (int l = 0; l < nl; ++l) {
    TRY(check_csr(&K[l], what));
    if (K[l].nrows != K[l].ncols) return fail(STOKES_ERR_INVALID_ARG, std::string(what) + ": operator not square");
    if (l + 1 < nl) {
      TRY(check_csr(&P[l], what));
      if (P[l].nrows != K[l].nrows || P[l].ncols != K[l + 1].nrows)
        return fail(STOKES_ERR_INVALID_ARG, std::string(what) + ": prolongator sizes");
    }
  }
  for (int l = 0; l < nl; ++l) {
    Level& lv = lvs[l];
    lv.n = K[l].nrows;
    lv.seg_off.assign(1, 0);
    HostCSR Kh;
    Kh.nrows = Kh.ncols = (int)lv.n;
    append_block(Kh, &K[l], 0);
    TRY(upload_csr(h, lv.K, Kh));
    if (l + 1 < nl) {
      HostCSR Ph;
      Ph.nrows = (int)lv.n;
      Ph.ncols = K[l + 1].nrows;
      append_block(Ph, &P[l], 0);
      lv.hasP = true;
      TRY(upload_csr(h, lv.P, Ph));
      TRY(upload_csr(h, lv.R, transpose(Ph)));
      // Jacobi diagonals
      std::vector<double> d(lv.n, 0.0);
      for (int i = 0; i < K[l].nrows; ++i)
        for (int64_t k = K[l].rowptr[i]; k < K[l].rowptr[i + 1]; ++k)
          if (K[l].col[k] == i) d[i] = K[l].val[k];
      for (auto& v : d) {
        if (!(v != 0.0)) return fail(STOKES_ERR_INVALID_ARG, std::string(what) + ": zero diagonal");
        v = 1.0 / v;
      }
      char* dv = nullptr;
      if (h->prec == STOKES_FP32) {
        std::vector<float> f(d.begin(), d.end());
        float* q = nullptr;
        TRY(upload(h, &q, f));
        dv = reinterpret_cast<char*>(q);
      } else {
        double* q = nullptr;
        TRY(upload(h, &q, d));
        dv = reinterpret_cast<char*>(q);
      }
      lv.dinv = dv;
      lv.jacobi = true;
      lv.relax = STOKES_RELAX_VANKA_KRYLOV;
      lv.krylov = true;
      lv.kmax = h->btp_steps;
      const int k = lv.kmax;
      lv.lds = 1 + k * (k + 1) + k;
      lv.ldp = kKrMaxSteps;
      std::vector<int64_t> cb, ce;
      std::vector<int> cs, sb{0}, se;
      for (int64_t r = 0; r < lv.n; r += 2048) {
        cb.push_back(r);
        ce.push_back(std::min<int64_t>(lv.n, r + 2048));
        cs.push_back(0);
      }
      se.push_back((int)cb.size());
      lv.kch.n = (int)cb.size();
      TRY(upload(h, &lv.kch.beg, cb));
      TRY(upload(h, &lv.kch.end, ce));
      TRY(upload(h, &lv.kch.seg, cs));
      TRY(upload(h, &lv.kch.sbeg, sb));
      TRY(upload(h, &lv.kch.send, se));
      char *V, *Z;
      TRY(dalloc(h, &V, (size_t)(k + 1) * lv.n * T));
      TRY(dalloc(h, &Z, (size_t)k * lv.n * T));
      lv.kV = V;
      lv.kZ = Z;
      TRY(dalloc(h, &lv.kS, (size_t)lv.lds));
      TRY(dalloc(h, &lv.kpart, (size_t)std::max(lv.kch.n, 1) * lv.ldp));
      TRY(dalloc(h, &lv.kcnt, 1));
      CK(cudaMemset(lv.kcnt, 0, sizeof(int)));
    } else {
      std::vector<double> inv;
      TRY(bordered_inverse(&K[l], nullptr, inv));
      std::vector<int> boff{0}, bn{K[l].nrows};
      std::vector<int64_t> koff{0};
      TRY(upload(h, &lv.coarse.boff, boff));
      TRY(upload(h, &lv.coarse.bn, bn));
      TRY(upload(h, &lv.coarse.koff, koff));
      TRY(upload(h, &lv.coarse.Kinv, inv));
      lv.coarse.nblocks = 1;
      lv.coarse.max_n = K[l].nrows;
      lv.coarse.kinv_elems = (int64_t)inv.size();
    }
    char *x, *b, *r, *ta, *tb;
    TRY(dalloc(h, &x, (size_t)lv.n * T));
    TRY(dalloc(h, &b, (size_t)lv.n * T));
    TRY(dalloc(h, &r, (size_t)lv.n * T));
    TRY(dalloc(h, &ta, (size_t)lv.n * T));
    TRY(dalloc(h, &tb, (size_t)lv.n * T));
    lv.x = x; lv.b = b; lv.r = r; lv.ta = ta; lv.tb = tb;
  }
  return STOKES_OK;
}

static int setup_btp(stokes_handle* h, const stokes_problem* p, int dim) {
  const stokes_btp* q = p->btp;
  if (!q) return fail(STOKES_ERR_INVALID_ARG, "BTP needs stokes_problem.btp");
  if (q->nlevels_a < 1 || !q->A || (q->nlevels_a > 1 && !q->PA) || !q->B)
    return fail(STOKES_ERR_INVALID_ARG, "btp: A hierarchy or B missing");
  const int64_t nu = p->field_off[dim], np = p->field_off[dim + 1] - nu;
  if (q->A[0].nrows != nu) return fail(STOKES_ERR_INVALID_ARG, "btp: A[0] is not the velocity block of K0");
  TRY(check_csr(q->B, "btp B"));
  if (q->B->nrows != np || q->B->ncols != nu) return fail(STOKES_ERR_INVALID_ARG, "btp: B sizes");
  TRY(setup_btp_levels(h, h->btpA, q->A, q->PA, q->nlevels_a, "btp A"));
  HostCSR Bh;
  Bh.nrows = (int)np;
  Bh.ncols = (int)nu;
  append_block(Bh, q->B, 0);
  TRY(upload_csr(h, h->btpB, Bh));
  if (q->Minv) {
    TRY(check_csr(q->Minv, "btp Minv"));
    if (q->Minv->nrows != np || q->Minv->ncols != np) return fail(STOKES_ERR_INVALID_ARG, "btp: Minv sizes");
    HostCSR Mh;
    Mh.nrows = Mh.ncols = (int)np;
    append_block(Mh, q->Minv, 0);
    TRY(upload_csr(h, h->btpMinv, Mh));
  } else {
    if (q->nlevels_m < 1 || !q->M || (q->nlevels_m > 1 && !q->PM))
      return fail(STOKES_ERR_INVALID_ARG, "btp: give the M hierarchy or Minv");
    if (q->M[0].nrows != np) return fail(STOKES_ERR_INVALID_ARG, "btp: M[0] size");
    TRY(setup_btp_levels(h, h->btpM, q->M, q->PM, q->nlevels_m, "btp M"));
  }
  char* tp = nullptr;
  TRY(dalloc(h, &tp, (size_t)3 * np * esz(h)));
  h->btp_tp = tp;
  return STOKES_OK;
}

static int setup_impl(stokes_handle* h, const stokes_problem* const* probs, int ninst, const stokes_params* prm) {
  const int dim = probs[0]->dim;
  h->dim = dim;
  h->disc = probs[0]->disc;
  h->prec = prm->precision;
  h->schedule = prm->schedule;
  h->nu1 = prm->nu1;
  h->nu2 = prm->nu2;
  h->eta_u = prm->eta_u;
  h->eta_p = prm->eta_p;
  if (h->prec != STOKES_FP32 && h->prec != STOKES_FP64) return fail(STOKES_ERR_INVALID_ARG, "precision");
  h->precond = prm->preconditioner;
  h->btp_steps = prm->btp_steps;
  h->factor_tcgen05 = prm->factor_tcgen05 != 0;
  if (h->precond != STOKES_PRECOND_DC && h->precond != STOKES_PRECOND_BTP)
    return fail(STOKES_ERR_INVALID_ARG, "unknown preconditioner");
  if (h->precond == STOKES_PRECOND_BTP) {
    if (ninst != 1) return fail(STOKES_ERR_INVALID_ARG, "BTP handles hold one instance");
    if (h->btp_steps < 1 || h->btp_steps > kKrMaxSteps) return fail(STOKES_ERR_INVALID_ARG, "btp_steps must be 1..4");
  }
  if (prm->nu1 < 0 || prm->nu2 < 0 || prm->schedule < 0 || prm->schedule > 2)
    return fail(STOKES_ERR_INVALID_ARG, "schedule or sweep counts");
  if (h->disc != STOKES_TH && h->disc != STOKES_SV) return fail(STOKES_ERR_INVALID_ARG, "disc must be TH or SV");
  for (int c = 0; c < 3; ++c) h->cheb_deg[c] = prm->cheb_deg[c];
  h->dlsc_sweeps = prm->dlsc_sweeps;
  h->mcg_deg = prm->mcg_deg;
  if (h->dlsc_sweeps < 0 || h->mcg_deg < 0 || h->cheb_deg[0] < 0 || h->cheb_deg[1] < 0 || h->cheb_deg[2] < 0)
    return fail(STOKES_ERR_INVALID_ARG, "negative Chebyshev degree or sweep count");
  int L = 0;
  for (int k = 0; k < ninst; ++k) {
    const stokes_problem* p = probs[k];
    if (!p || p->dim != dim || p->disc != h->disc || p->nlevels < 2 || !p->K || !p->P || !p->patches ||
        !p->field_off || !p->coarse_null || !p->dirichlet)
      return fail(STOKES_ERR_INVALID_ARG, "problem " + std::to_string(k) + ": missing fields or mismatched dim/disc");
    if (dim != 2 && dim != 3) return fail(STOKES_ERR_INVALID_ARG, "dim must be 2 or 3");
    h->inst_levels.push_back(p->nlevels);
    L = std::max(L, (int)p->nlevels);
    for (int l = 0; l < p->nlevels; ++l) {
      TRY(check_csr(&p->K[l], "K"));
      const int64_t* off = p->field_off + (size_t)l * (dim + 2);
      if (off[0] != 0 || off[dim + 1] != p->K[l].nrows || p->K[l].nrows != p->K[l].ncols)
        return fail(STOKES_ERR_INVALID_ARG, "field_off/K size mismatch on level " + std::to_string(l));
      for (int c = 0; c <= dim; ++c)
        if (off[c + 1] < off[c]) return fail(STOKES_ERR_INVALID_ARG, "field_off decreases");
    }
    for (int l = 0; l + 1 < p->nlevels; ++l) {
      TRY(check_csr(&p->P[l], "P"));
      if (p->P[l].nrows != p->K[l].nrows || p->P[l].ncols != p->K[l + 1].nrows)
        return fail(STOKES_ERR_INVALID_ARG, "P size mismatch on level " + std::to_string(l));
    }
    if (h->disc == STOKES_SV) {
      if (!p->R0p || !p->Mcg) return fail(STOKES_ERR_INVALID_ARG, "Scott-Vogelius problems need R0p and Mcg");
      TRY(check_csr(p->R0p, "R0p"));
      TRY(check_csr(p->Mcg, "Mcg"));
      const int64_t* o0 = p->field_off;
      const int64_t* o1 = p->field_off + (dim + 2);
      if (o1[dim] != o0[dim] || p->R0p->ncols != o0[dim + 1] - o0[dim] || p->R0p->nrows != o1[dim + 1] - o1[dim] ||
          p->Mcg->nrows != p->R0p->nrows || p->Mcg->ncols != p->Mcg->nrows)
        return fail(STOKES_ERR_INVALID_ARG, "R0p/Mcg sizes do not match levels 0 and 1");
      if (!(p->mcg_lo > 0 && p->mcg_hi > p->mcg_lo)) return fail(STOKES_ERR_INVALID_ARG, "mcg interval");
      if (k > 0 && (p->mcg_lo != probs[0]->mcg_lo || p->mcg_hi != probs[0]->mcg_hi))
        return fail(STOKES_ERR_INVALID_ARG, "instances must share the Mcg interval");
    }
  }
  h->L = L;
  h->lv.resize(L);
  std::vector<double> omega(L, 1.0);
  std::vector<int> relaxk(L, STOKES_RELAX_VANKA);
  for (int l = 0; l + 1 < L; ++l) {
    if (prm->omega) omega[l] = prm->omega[l];
    if (prm->relax) relaxk[l] = prm->relax[l];
    if (relaxk[l] != STOKES_RELAX_VANKA && relaxk[l] != STOKES_RELAX_DLSC && relaxk[l] != STOKES_RELAX_VANKA_KRYLOV)
      return fail(STOKES_ERR_INVALID_ARG, "unknown relaxation");
    if (relaxk[l] == STOKES_RELAX_VANKA_KRYLOV && std::max(prm->nu1, prm->nu2) > kKrMaxSteps)
      return fail(STOKES_ERR_INVALID_ARG, "Krylov-wrapped relaxation: at most 4 inner steps (nu1, nu2)");
    if (relaxk[l] == STOKES_RELAX_DLSC) {
      for (int k = 0; k < ninst; ++k) {
        if (probs[k]->nlevels - 1 <= l) continue;
        if (!probs[k]->lambda_A || !probs[k]->lambda_S)
          return fail(STOKES_ERR_INVALID_ARG, "DLSC needs lambda_A and lambda_S");
        if (l == 0 && !probs[k]->Mu_diag)
          return fail(STOKES_ERR_INVALID_ARG, "DLSC on level 0 needs Mu_diag (diagonal of the velocity mass matrix)");
        if (probs[k]->lambda_A[l] != probs[0]->lambda_A[l] || probs[k]->lambda_S[l] != probs[0]->lambda_S[l])
          return fail(STOKES_ERR_INVALID_ARG, "DLSC instances must share their Chebyshev bounds");
      }
    }
  }
  const size_t T = esz(h);
  // segment offsets per level
  for (int l = 0; l < L; ++l) {
    Level& lv = h->lv[l];
    lv.seg_off.assign(ninst, -1);
    int64_t n = 0;
    for (int k = 0; k < ninst; ++k)
      if (probs[k]->nlevels > l) {
        lv.seg_off[k] = n;
        n += probs[k]->K[l].nrows;
      }
    lv.n = n;
    lv.omega = omega[l];
    lv.relax = relaxk[l];
    if (n >= (int64_t(1) << 31)) return fail(STOKES_ERR_INVALID_ARG, "level too large for int32 indices");
  }
  for (int l = 0; l < L; ++l) {
    Level& lv = h->lv[l];
    // K_l block diagonal over instances
    HostCSR K;
    K.nrows = K.ncols = (int)lv.n;
    for (int k = 0; k < ninst; ++k)
      if (probs[k]->nlevels > l) append_block(K, &probs[k]->K[l], lv.seg_off[k]);
    TRY(upload_csr(h, lv.K, K));
    // P_l: level l+1 -> l (zero rows for instances ending at l)
    if (l + 1 < L) {
      const Level& lc = h->lv[l + 1];
      HostCSR P;
      P.nrows = (int)lv.n;
      P.ncols = (int)lc.n;
      bool ident = true;
      for (int k = 0; k < ninst; ++k) {
        if (probs[k]->nlevels <= l) continue;
        if (probs[k]->nlevels > l + 1) {
          append_block(P, &probs[k]->P[l], lc.seg_off[k]);
          ident = ident && is_identity(&probs[k]->P[l]);
        } else {
          append_zero_rows(P, probs[k]->K[l].nrows);
          ident = false;
        }
      }
      lv.hasP = true;
      lv.Pident = ident && l == 0;
      TRY(upload_csr(h, lv.P, P));
      const HostCSR R = transpose(P);
      TRY(upload_csr(h, lv.R, R));
      // levels >= 3: R (b - K x) as R b - (R K) x in one launch where R K has
      // no more entries than K and R together (on levels 1 and 2 the
      // sliced-ELLPACK / row-block residual and restriction measured faster)
      if (l >= 3) {
        HostCSR RK = csr_product(R, K, nullptr);
        if (RK.col.size() <= K.col.size() + R.col.size()) {
          TRY(upload_csr(h, lv.RK, RK));
          lv.hasRK = true;
        }
      }
    }
    // coarsest blocks of the instances ending at l
    std::vector<int> boff, bn;
    std::vector<int64_t> koff;
    std::vector<double> kinv;
    for (int k = 0; k < ninst; ++k) {
      if (probs[k]->nlevels != l + 1) continue;
      std::vector<double> inv;
      TRY(bordered_inverse(&probs[k]->K[l], probs[k]->coarse_null, inv));
      boff.push_back((int)lv.seg_off[k]);
      bn.push_back(probs[k]->K[l].nrows);
      koff.push_back((int64_t)kinv.size());
      kinv.insert(kinv.end(), inv.begin(), inv.end());
      lv.coarse.max_n = std::max(lv.coarse.max_n, probs[k]->K[l].nrows);
    }
    lv.coarse.nblocks = (int)boff.size();
    if (lv.coarse.nblocks) {
      TRY(upload(h, &lv.coarse.boff, boff));
      TRY(upload(h, &lv.coarse.bn, bn));
      TRY(upload(h, &lv.coarse.koff, koff));
      TRY(upload(h, &lv.coarse.Kinv, kinv));
      lv.coarse.kinv_elems = (int64_t)kinv.size();
    }
    if (l + 1 < L && relaxk[l] == STOKES_RELAX_DLSC) {
      TRY(setup_dlsc(h, lv, probs, ninst, l, dim));
      continue;
    }
    // Vanka patches of the instances relaxing on l, validated, in original order
    std::vector<int> optr{0}, odof, onv, onp;
    bool shared = true;
    const int align = 16 / (int)T;
    for (int k = 0; k < ninst; ++k) {
      const stokes_problem* p = probs[k];
      if (p->nlevels - 1 <= l) continue;
      const stokes_patches* pa = &p->patches[l];
      const int64_t* off = p->field_off + (size_t)l * (dim + 2);
      if (pa->npatch < 0 || (pa->npatch > 0 && (!pa->ptr || !pa->dof || !pa->nvel || !pa->npres)))
        return fail(STOKES_ERR_INVALID_ARG, "patches: null arrays");
      bool sh = components_share_block(&p->K[l], off, dim);
      for (int i = 0; i < pa->npatch; ++i) {
        const int m = pa->nvel[(size_t)i * dim];
        const int np = pa->npres[i];
        for (int c = 1; c < dim; ++c)
          if (pa->nvel[(size_t)i * dim + c] != m)
            return fail(STOKES_ERR_INVALID_ARG, "patches: components must hold the same number of DoFs");
        if (np < 1 || np > 4) return fail(STOKES_ERR_INVALID_ARG, "patches: 1..4 pressure seeds per patch");
        if (m < 1 || m > 512) return fail(STOKES_ERR_INVALID_ARG, "patches: 1..512 velocity DoFs per component");
        const int64_t b0 = pa->ptr[i], b1 = pa->ptr[i + 1];
        if (b1 - b0 != (int64_t)dim * m + np) return fail(STOKES_ERR_INVALID_ARG, "patches: ptr does not match nvel/npres");
        for (int c = 0; c <= dim; ++c) {
          const int cnt = c < dim ? m : np;
          const int64_t s0 = b0 + (int64_t)c * m;
          for (int a = 0; a < cnt; ++a) {
            const int g = pa->dof[s0 + a];
            if (g < off[c] || g >= off[c + 1])
              return fail(STOKES_ERR_INVALID_ARG, "patches: DoF outside its field range");
            if (a > 0 && g <= pa->dof[s0 + a - 1]) return fail(STOKES_ERR_INVALID_ARG, "patches: DoFs not ascending");
            if (l == 0 && p->dirichlet[g]) return fail(STOKES_ERR_INVALID_ARG, "patches: Dirichlet DoF in a patch");
            if (c > 0 && c < dim && g - off[c] != pa->dof[b0 + a] - off[0]) sh = false;
          }
        }
        for (int64_t q = b0; q < b1; ++q) odof.push_back((int)(pa->dof[q] + lv.seg_off[k]));
        optr.push_back((int)odof.size());
        onv.push_back(m);
        onp.push_back(np);
      }
      shared = shared && sh;
    }
    if (onv.empty()) continue;
    // storage order: the bulk-copy bins by m (<= 6, 20, 32, 64, 96), then the rest;
    // a bin whose smallest tile (4 patches per warp group, 3 stages) would not
    // fit in shared memory hands its patches to the CTA-per-patch kernel
    const int npatch = (int)onv.size();
    const int nblk0 = shared ? 1 : dim;
    bool bin_ok[kTmaBins];
    for (int b = 0; b < kTmaBins; ++b) {
      int64_t maxblk = 0;
      for (int i = 0; i < npatch; ++i)
        if (vanka_tma_bin_of(onv[i]) == b) {
          const int64_t m = onv[i], np = onp[i];
          const int64_t pkp = (m * (m + 1) / 2 + align - 1) / align * align;
          maxblk = std::max(maxblk, (nblk0 * pkp + dim * m * np + np * np + align) * (int64_t)T);
        }
      const int ppw = vanka_tma_bin_ppw(b);
      bin_ok[b] = 3 * 4 * ppw * maxblk <= 160 * 1024;
    }
    // a nearly empty bin (e.g. the few corner patches below m = 8) joins the
    // next larger usable bin, whose kernel handles any smaller m: one launch less
    int bin_cnt[kTmaBins] = {0};
    for (int i = 0; i < npatch; ++i) {
      const int b = vanka_tma_bin_of(onv[i]);
      if (b >= 0) bin_cnt[b]++;
    }
    int bin_map[kTmaBins];
    for (int b = kTmaBins - 1; b >= 0; --b) {
      bin_map[b] = bin_ok[b] ? b : -1;
      if (bin_ok[b] && b + 1 < kTmaBins && bin_map[b + 1] >= 0) {
        const int up = bin_map[b + 1];
        if (bin_cnt[b] < std::max(64, bin_cnt[up] / 4)) {
          bin_map[b] = up;
          bin_cnt[up] += bin_cnt[b];
        }
      }
    }
    auto bin_of = [&](int m) {
      const int b = vanka_tma_bin_of(m);
      return b >= 0 ? bin_map[b] : -1;
    };
    std::vector<int> order;
    int bin_start[kTmaBins + 1];
    for (int b = 0; b < kTmaBins; ++b) {
      bin_start[b] = (int)order.size();
      for (int i = 0; i < npatch; ++i)
        if (bin_of(onv[i]) == b) order.push_back(i);
    }
    bin_start[kTmaBins] = (int)order.size();
    const int nsmall = (int)order.size();
    // the rest (tiled blocks) by descending m: the persistent apply deals
    // them round robin to its warps
    for (int i = 0; i < npatch; ++i)
      if (bin_of(onv[i]) < 0) order.push_back(i);
    std::stable_sort(order.begin() + nsmall, order.end(), [&](int a, int b) { return onv[a] > onv[b]; });
    std::vector<int> pptr{0}, pdof, pnv, pnp, small, large, stor(npatch);
    std::vector<int64_t> foff;
    int64_t fac = 0;
    const int nblk = shared ? 1 : dim;
    int max_m = 0, max_np = 0, max_m_large = 0, max_np_small = 0;
    for (int si = 0; si < npatch; ++si) {
      const int i = order[si];
      stor[i] = si;
      for (int q = optr[i]; q < optr[i + 1]; ++q) pdof.push_back(odof[q]);
      pptr.push_back((int)pdof.size());
      const int64_t m = onv[i], np = onp[i];
      pnv.push_back((int)m);
      pnp.push_back((int)np);
      foff.push_back(fac);
      // blocks start 16-byte aligned; bulk-copy bins packed, the rest tiled
      const int64_t pkp = si < nsmall ? (m * (m + 1) / 2 + align - 1) / align * align : tiled_block_elems((int)m);
      int64_t sz = nblk * pkp + dim * m * np + np * np;
      fac += (sz + align - 1) / align * align;
      (si < nsmall ? small : large).push_back(si);
      max_m = std::max(max_m, (int)m);
      max_np = std::max(max_np, (int)np);
      if (si >= nsmall) max_m_large = std::max(max_m_large, (int)m);
      else max_np_small = std::max(max_np_small, (int)np);
    }
    foff.push_back(fac);  // sentinel
    // transpose map: DoF -> slots, in ascending ORIGINAL patch order
    std::vector<int> tptr(lv.n + 1, 0), tslot(pdof.size());
    for (int g : pdof) tptr[g + 1]++;
    for (int64_t j = 0; j < lv.n; ++j) tptr[j + 1] += tptr[j];
    std::vector<int> pos(tptr.begin(), tptr.end() - 1);
    for (int i = 0; i < npatch; ++i) {
      const int si = stor[i];
      for (int q = pptr[si]; q < pptr[si + 1]; ++q) tslot[pos[pdof[q]]++] = q;
    }
    // per-patch metadata for the bulk-copy tiles
    std::vector<int4> meta(npatch);
    for (int si = 0; si < npatch; ++si)
      meta[si] = make_int4(pptr[si], pnv[si] | (pnp[si] << 16), (int)(uint32_t)(foff[si] & 0xffffffffu),
                           (int)(foff[si] >> 32));
    DevPatches& dp = lv.pat;
    dp.npatch = npatch;
    dp.dim = dim;
    dp.shared = shared ? 1 : 0;
    dp.tcgen05 = h->factor_tcgen05 ? 1 : 0;
    dp.nsmall = (int)small.size();
    dp.nlarge = (int)large.size();
    dp.max_m = max_m;
    dp.max_np = max_np;
    dp.max_m_large = max_m_large;
    dp.fac_elems = fac;
    dp.nslots = (int64_t)pdof.size();
    // bulk-copy tiles per bin: about 8 KB of factors per stage (at least one
    // patch per consumer lane group), 3 stages
    for (int b = 0; b < kTmaBins; ++b) {
      TmaBin& bn = dp.bins[b];
      bn.start = bin_start[b];
      bn.count = bin_start[b + 1] - bin_start[b];
      if (bn.count == 0) continue;
      int64_t maxblk = 0;
      for (int si = bn.start; si < bn.start + bn.count; ++si) {
        maxblk = std::max(maxblk, (foff[si + 1] - foff[si]) * (int64_t)T);
        bn.max_np = std::max(bn.max_np, pnp[si]);
      }
      const int ppw = vanka_tma_bin_ppw(b);  // patches per warp at a time
      bn.tp = (int)std::max<int64_t>(4 * ppw, std::min<int64_t>(64, 8192 / std::max<int64_t>(maxblk, 1)));
    }
    std::vector<int> pdof_pad(pdof);
    pdof_pad.resize(pdof.size() + 8, 0);  // bulk copies may read up to 16 bytes past the last list
    TRY(upload(h, &dp.ptr, pptr));
    TRY(upload(h, &dp.dof, pdof_pad));
    TRY(upload(h, &dp.nvel, pnv));
    TRY(upload(h, &dp.npres, pnp));
    TRY(upload(h, &dp.foff, foff));
    TRY(upload(h, &dp.small, small));
    TRY(upload(h, &dp.large, large));
    TRY(upload(h, &dp.tptr, tptr));
    {
      // the apply writes slot q to yp[pdst[q]]: DoF-major, so the scatter reads each DoF's
      // solutions contiguously (same order as the transpose map)
      std::vector<int> pdst(pdof.size() + 8, 0);
      for (size_t t = 0; t < tslot.size(); ++t) pdst[tslot[t]] = (int)t;
      TRY(upload(h, &dp.pdst, pdst));
    }
    TRY(upload(h, &dp.meta, meta));
    TRY(dalloc(h, &dp.err, 1));
    CK(cudaMemset(dp.err, 0, sizeof(int)));
    h->err_flags.push_back(dp.err);
    {
      int nsm = 0, dev = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
      for (int b = 0; b < kTmaBins; ++b) {
        TmaBin& bn = dp.bins[b];
        if (bn.count == 0) continue;
        // a 2-stage ring when it keeps clearly more CTAs (consumer warps) per SM
        const int tp = bn.tp;
        if (!configure_bin(dp, bn, b, tp, 3, foff, pptr, T, nsm))
          return fail(STOKES_ERR_INVALID_ARG, "patch tiles do not fit on an SM");
        const int nb3 = bn.grid;
        TmaBin b2 = bn;
        if (configure_bin(dp, b2, b, tp, 2, foff, pptr, T, nsm) && b2.grid * 2 >= nb3 * 3) bn = b2;
      }
      lv.hfoff = foff;
      lv.hpptr = pptr;
      dp.use_tma = nsmall > 0;
    }
    // factorisation order: warp bins; then FP32: tensor-core sweep grouped by
    // tile rows (shared memory), the rest in global scratch; FP64: blocks that
    // fit in shared memory, then the rest
    {
      int optin = 0, dev = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      std::vector<int> fl, fg, fw[3], ft[kTcMaxSmemRows + 1];
      int msm = 0, glob_rows = 0;
      for (int si = 0; si < npatch; ++si) {
        const int wb = vanka_factor_warp_bin(pnv[si]);
        const int rows = tile_rows(pnv[si]);
        if (wb >= 0) {
          fw[wb].push_back(si);
        } else if (T == 4) {
          if (rows <= kTcMaxSmemRows &&
              vanka_factor_tc_smem(dim, rows, max_np, false,
                                   h->factor_tcgen05 && rows >= kUmmaMinRows && rows <= kUmmaMaxRowsFac) <=
                  (size_t)optin) {
            ft[rows].push_back(si);
          } else {
            fg.push_back(si);
            glob_rows = std::max(glob_rows, rows);
          }
        } else if (vanka_factor_smem(dim, pnv[si], max_np, T, false) <= (size_t)optin) {
          fl.push_back(si);
          msm = std::max(msm, pnv[si]);
        } else {
          fg.push_back(si);
        }
      }
      if (T == 4) {
        for (int rows = 1; rows <= kTcMaxSmemRows; ++rows) {
          dp.nfac_tc[rows] = (int)ft[rows].size();
          fl.insert(fl.end(), ft[rows].begin(), ft[rows].end());
        }
        dp.tc_glob_rows = glob_rows;
      } else {
        dp.nfac_smem = (int)fl.size();
        dp.max_m_fac_smem = msm;
      }
      fl.insert(fl.end(), fg.begin(), fg.end());
      for (int b = 2; b >= 0; --b) {
        dp.nfac_warp[b] = (int)fw[b].size();
        fl.insert(fl.begin(), fw[b].begin(), fw[b].end());
      }
      TRY(upload(h, &dp.fac_list, fl));
      if (!fg.empty()) {
        size_t scr_bytes;
        if (T == 4) {
          if (vanka_factor_tc_smem(dim, glob_rows, max_np, true, false) > (size_t)optin)
            return fail(STOKES_ERR_INVALID_ARG, "patch too large for the factorisation kernel");
          scr_bytes = (size_t)dp.fac_chunk * ((size_t)glob_rows * (glob_rows + 1) / 2 + glob_rows) * kTileElems * 4;
        } else {
          if (vanka_factor_smem(dim, max_m, max_np, T, true) > (size_t)optin)
            return fail(STOKES_ERR_INVALID_ARG, "patch too large for the factorisation kernel");
          scr_bytes = (size_t)dp.fac_chunk * max_m * max_m * T;
        }
        char* scr = nullptr;
        TRY(dalloc(h, &scr, scr_bytes));
        dp.fac_scratch = scr;
      }
      // apply of the tiled patches: per consumer warp a ring that holds U |
      // S^-1 and the output positions at once, plus two tiles of prefetch
      if (!large.empty()) {
        if (dim * max_m_large + max_np + 6 > kTileElems)
          return fail(STOKES_ERR_INVALID_ARG, "patch too large for the tiled apply");
        int nus = 0;
        for (int si : large) {
          const int64_t L = (int64_t)dim * pnv[si] * pnp[si] + (int64_t)pnp[si] * pnp[si];
          nus = std::max(nus, (int)((L + kTileElems - 1) / kTileElems));
        }
        dp.tiles_nodes = 32 * tile_rows(max_m_large);
        int nsm = 0;
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        int stages = std::max(4, nus + 3);
        int per_sm = 0;
        for (; stages >= nus + 1; --stages) {
          if (vanka_tiles_smem(stages, dp.tiles_nodes, dim, T) > (size_t)optin) continue;
          per_sm = vanka_tiles_blocks_per_sm(stages, dp.tiles_nodes, dim, max_np, T);
          if (per_sm > 0) break;
        }
        if (per_sm <= 0) return fail(STOKES_ERR_INVALID_ARG, "tiled patches do not fit on an SM");
        dp.tiles_stages = stages;
        const int want = (int)((large.size() + 3) / 4);  // four consumer warps per CTA
        dp.tiles_grid = std::max(1, std::min(want, per_sm * nsm));
      }
    }
    char* facp = nullptr;
    TRY(dalloc(h, &facp, (size_t)fac * T));
    dp.fac = facp;
    char* yp = nullptr;
    TRY(dalloc(h, &yp, (size_t)dp.nslots * T));
    lv.yp = yp;
    lv.has_patches = true;
  }
  // level vectors
  for (int l = 0; l < L; ++l) {
    Level& lv = h->lv[l];
    char *x, *b, *r, *ta, *tb;
    TRY(dalloc(h, &x, (size_t)lv.n * T));
    TRY(dalloc(h, &b, (size_t)lv.n * T));
    TRY(dalloc(h, &r, (size_t)lv.n * T));
    TRY(dalloc(h, &ta, (size_t)lv.n * T));
    TRY(dalloc(h, &tb, (size_t)lv.n * T));
    lv.x = x; lv.b = b; lv.r = r; lv.ta = ta; lv.tb = tb;
  }
  for (int l = 0; l + 1 < L; ++l)
    if (h->lv[l].relax == STOKES_RELAX_VANKA_KRYLOV) TRY(setup_krylov_relax(h, h->lv[l], probs, ninst, l));
  if (h->disc == STOKES_SV) TRY(setup_sv(h, probs, ninst, dim));
  if (h->precond == STOKES_PRECOND_BTP) TRY(setup_btp(h, probs[0], dim));
  if (h->prec == STOKES_FP32) TRY(dalloc(h, &h->x0_64, (size_t)h->lv[0].n));
  if (!h->d0buf) TRY(dalloc(h, &h->d0buf, (size_t)h->lv[0].n));
  // level-0 row kinds and Dirichlet mask
  {
    std::vector<uint8_t> kind(h->lv[0].n), dir(h->lv[0].n);
    for (int k = 0; k < ninst; ++k) {
      const stokes_problem* p = probs[k];
      const int64_t* off = p->field_off;
      const int64_t o = h->lv[0].seg_off[k];
      for (int64_t i = 0; i < p->K[0].nrows; ++i) {
        dir[o + i] = p->dirichlet[i] ? 1 : 0;
        kind[o + i] = p->dirichlet[i] ? 2 : (i >= off[dim] ? 1 : 0);
      }
    }
    TRY(upload(h, &h->kind0, kind));
    TRY(upload(h, &h->dir0, dir));
  }
  // FGMRES chunks (never straddling an instance): 512 rows (two per thread
  // of a 256-thread block) for the updates, 2048 rows for the dot products,
  // whose block reductions then cost a small share of their FP64 work
  for (int t = 0; t < 2; ++t) {
    std::vector<int64_t> cb, ce;
    std::vector<int> cs, sb(ninst, 0), se(ninst, 0);
    const int64_t CH = t == 0 ? 512 : 2048;
    for (int k = 0; k < ninst; ++k) {
      const int64_t o = h->lv[0].seg_off[k], n = probs[k]->K[0].nrows;
      sb[k] = (int)cb.size();
      for (int64_t s = 0; s < n; s += CH) {
        cb.push_back(o + s);
        ce.push_back(o + std::min(n, s + CH));
        cs.push_back(k);
      }
      se[k] = (int)cb.size();
    }
    if (t == 0) {
      h->nchunks = (int)cb.size();
      TRY(upload(h, &h->cbeg, cb));
      TRY(upload(h, &h->cend, ce));
      TRY(upload(h, &h->cseg, cs));
    } else {
      h->ndchunks = (int)cb.size();
      TRY(upload(h, &h->dbeg, cb));
      TRY(upload(h, &h->dend, ce));
      TRY(upload(h, &h->sd_beg, sb));
      TRY(upload(h, &h->sd_end, se));
      h->arch.n = h->ndchunks;
      h->arch.beg = h->dbeg;
      h->arch.end = h->dend;
      h->arch.sbeg = h->sd_beg;
      h->arch.send = h->sd_end;
      TRY(upload(h, &h->arch.seg, cs));
      std::vector<int> zero(ninst, 0);
      TRY(upload(h, &h->arcnt, zero));
    }
  }
  return STOKES_OK;
}

int stokes_setup(const stokes_problem* const* probs, int32_t ninstances, const stokes_params* params,
                 void* cuda_stream, stokes_handle** out) {
  if (!out) return fail(STOKES_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!probs || ninstances < 1 || !params) return fail(STOKES_ERR_INVALID_ARG, "no problems or params");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(STOKES_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  stokes_handle* h = new stokes_handle();
  h->ninst = ninstances;
  if (cuda_stream) {
    h->st = reinterpret_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete h;
      return fail(STOKES_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    h->own_stream = true;
    if (cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess) {
      stokes_destroy(h);
      return fail(STOKES_ERR_CUDA, "cudaEventCreate failed");
    }
  }
  e = cudaEventCreateWithFlags(&h->fj.fork, cudaEventDisableTiming);
  for (int k = 0; k < kForkMax && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&h->fj.side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->fj.join[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    stokes_destroy(h);
    return fail(STOKES_ERR_CUDA, std::string("side streams: ") + cudaGetErrorString(e));
  }
  e = vanka_prepare_kernels();
  if (e != cudaSuccess) {
    stokes_destroy(h);
    return fail(STOKES_ERR_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
  }
  int rc = setup_impl(h, probs, ninstances, params);
  if (rc != STOKES_OK) {
    stokes_destroy(h);
    return rc;
  }
  *out = h;
  return STOKES_OK;
}

int stokes_factor_patches(stokes_handle* h, int64_t* nsingular) {
  if (!h) return fail(STOKES_ERR_INVALID_ARG, "null handle");
  TRY(join_in(h));
  if (!h->dsing) TRY(dalloc(h, &h->dsing, 1));
  int* dsing = h->dsing;
  CK(cudaMemsetAsync(dsing, 0, sizeof(int), h->st));
  // the levels are independent (own factors and scratch): each runs on a
  // side stream, forked from and joined back to the handle's stream, so the
  // latency-bound launches of the small levels overlap the large ones
  CK(cudaEventRecord(h->fj.fork, h->st));
  bool used[kForkMax] = {};
  for (int l = 0; l < h->L; ++l) {
    Level& lv = h->lv[l];
    if (!lv.has_patches) continue;
    const int k = l % kForkMax;
    cudaStream_t s = h->fj.side[k];
    if (!used[k]) {
      CK(cudaStreamWaitEvent(s, h->fj.fork, 0));
      used[k] = true;
    }
    if (h->prec == STOKES_FP32) CK(vanka_factor<float>(lv.pat, lv.K, dsing, s));
    else CK(vanka_factor<double>(lv.pat, lv.K, dsing, s));
  }
  for (int k = 0; k < kForkMax; ++k)
    if (used[k]) {
      CK(cudaEventRecord(h->fj.join[k], h->fj.side[k]));
      CK(cudaStreamWaitEvent(h->st, h->fj.join[k], 0));
    }
  int ns = 0;
  CK(cudaMemcpyAsync(&ns, dsing, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (nsingular) *nsingular = ns;
  // a bounded wait of the tensor-core factorisation that ran out leaves
  // unusable factors (the same flags as the bulk-copy pipelines)
  TRY(check_pipeline_errors(h));
  h->factored = true;
  if (ns > 0) return fail(STOKES_ERR_SINGULAR_PATCH, std::to_string(ns) + " singular patches");
  return STOKES_OK;
}

int stokes_vcycle(stokes_handle* h, const double* r_dev, double* z_dev) {
  if (!h || !r_dev || !z_dev) return fail(STOKES_ERR_INVALID_ARG, "null argument");
  if (!h->factored && h->precond == STOKES_PRECOND_DC) return fail(STOKES_ERR_STATE, "stokes_factor_patches must run first");
  if ((const void*)r_dev == (void*)z_dev) return fail(STOKES_ERR_INVALID_ARG, "r and z alias");
  cudaGraphExec_t g;
  TRY(join_in(h));
  TRY(cycle_graph(h, r_dev, z_dev, &g));
  CK(cudaGraphLaunch(g, h->st));
  h->launches += h->cycle_launches;
  return join_out(h);
}

double stokes_cycle_bytes(const stokes_handle* hc) {
  stokes_handle* h = const_cast<stokes_handle*>(hc);
  if (!h) return 0.0;
  h->led = Ledger();
  h->led.count = true;
  run_cycle(h, nullptr, reinterpret_cast<double*>(16));
  const double b = h->led.bytes;
  h->led.count = false;
  return b;
}

double stokes_sweep_factor_bytes(const stokes_handle* h, int32_t l) {
  if (!h || l < 0 || l >= h->L || !h->lv[l].has_patches) return 0.0;
  return double(h->lv[l].pat.fac_elems) * esz(h);
}

}  // extern "C"

// ------------------------------------------------------------- FGMRES
namespace {

// The bulk-copy pipelines record a flag instead of waiting forever; a set
// flag means a result is unusable.
int check_pipeline_errors(stokes_handle* h) {
  for (int* f : h->err_flags) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, f, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (e) return fail(STOKES_ERR_CUDA, "a bulk-copy pipeline wait timed out (flag " + std::to_string(e) + ")");
  }
  return STOKES_OK;
}

int ensure_krylov(stokes_handle* h, int m) {
  if (h->krylov_m >= m && h->V) return STOKES_OK;
  if (h->ninst > 1024) return fail(STOKES_ERR_INVALID_ARG, "at most 1024 instances per handle");
  const int64_t n = h->lv[0].n;
  const int ni = h->ninst;
  h->krylov_m = m;
  h->ldh = m + 2;
  h->ldp = m + 2;
  TRY(dalloc(h, &h->V, (size_t)(m + 1) * n));
  TRY(dalloc(h, &h->Z, (size_t)m * n));
  TRY(dalloc(h, &h->w, (size_t)n));
  TRY(dalloc(h, &h->partial, (size_t)h->nchunks * h->ldp));
  TRY(dalloc(h, &h->hd, (size_t)ni * h->ldh));
  TRY(dalloc(h, &h->yd, (size_t)ni * h->ldh));
  TRY(dalloc(h, &h->actd, (size_t)ni));
  FgState& f = h->fg;
  TRY(dalloc(h, &f.H, (size_t)ni * (m + 1) * m));
  TRY(dalloc(h, &f.cs, (size_t)ni * m));
  TRY(dalloc(h, &f.sn, (size_t)ni * m));
  TRY(dalloc(h, &f.g, (size_t)ni * (m + 1)));
  TRY(dalloc(h, &f.bnorm, (size_t)ni));
  TRY(dalloc(h, &f.scale, (size_t)ni));
  TRY(dalloc(h, &f.y, (size_t)ni * h->ldh));
  TRY(dalloc(h, &f.run, (size_t)ni));
  TRY(dalloc(h, &f.its, (size_t)ni));
  TRY(dalloc(h, &f.kcol, (size_t)ni));
  TRY(dalloc(h, &f.err, 1));
  TRY(dalloc(h, &f.stat, (size_t)m + 1));
  if (h->hstat) cudaFreeHost(h->hstat);
  CK(cudaHostAlloc(reinterpret_cast<void**>(&h->hstat), sizeof(int) * (m + 1), cudaHostAllocDefault));
  h->ev_iter.resize(m);
  for (auto& e : h->ev_iter)
    if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  for (auto& kv : h->iter_graphs) cudaGraphExecDestroy(kv.second);
  h->iter_graphs.clear();
  return STOKES_OK;
}

// per-segment dots h[s][0..ncols) = V_k . w  (fresh or accumulated)
int seg_dots(stokes_handle* h, const double* V, int64_t ldv, int ncols, const double* w, int accumulate) {
  CK(multidot_partial(h->ndchunks, h->dbeg, h->dend, ncols, V, ldv, w, h->partial, h->ldp, h->st));
  CK(multidot_finish(h->ninst, h->sd_beg, h->sd_end, ncols, h->partial, h->ldp, h->hd, h->ldh, accumulate, h->st));
  return STOKES_OK;
}

// An FP32 DC cycle inside FGMRES reads its input in FP32 from lv[0].b: the
// kernel that forms each Krylov vector writes that copy too, so the cycle
// needs no FP64-to-FP32 conversion launch.
bool r32_input(const stokes_handle* h) { return h->prec == STOKES_FP32 && h->precond == STOKES_PRECOND_DC; }
float* r32_out(stokes_handle* h) { return r32_input(h) ? reinterpret_cast<float*>(h->lv[0].b) : nullptr; }

// One Arnoldi step j (Sec. 4, right-preconditioned flexible GMRES):
// z_j = M_dc^-1 v_j (the DC cycle), w = K0 z_j, classical Gram-Schmidt twice,
// device-side Givens update and v_{j+1} = w / ||w|| for running instances;
// the running flag lands in pinned host memory (hstat[j]).
int arnoldi_step(stokes_handle* h, int j, double rtol, int maxit) {
  const int64_t n = h->lv[0].n;
  const int ni = h->ninst;
  Level& L0 = h->lv[0];
  double* vj = h->V + (size_t)j * n;
  double* zj = h->Z + (size_t)j * n;
  h->r32_ready = r32_input(h);
  const int rc0 = run_cycle(h, vj, zj);
  h->r32_ready = false;
  TRY(rc0);
  CK((spmv<double, double, double, double, double>(L0.K, L0.K.v64, zj, zj, h->w, SPMV_SET, 0, 0, nullptr, h->st)));
  // classical Gram-Schmidt twice: h1 = V^T w, w -= V h1, h2 = V^T w,
  // w -= V h2, then ||w||^2 (a second pass is needed at nearly every step:
  // with a good preconditioner w = K0 z_j lies mostly in span V)
  const int nc = j + 1;
  if (nc <= kArMaxCols) {
    // fused passes: h1 -> hd, h2 -> yd, then the Givens update
    CK(ar_dots(h->arch, nc, h->V, n, h->w, h->partial, h->ldp, h->arcnt, h->hd, h->ldh, h->fg.stat + j, h->st));
    CK(ar_axpy_dots(h->arch, nc, h->V, n, h->hd, h->ldh, h->w, h->partial, h->ldp, h->arcnt, h->yd, h->st));
    CK(ar_axpy_norm_update(h->arch, nc, h->V, n, h->hd, h->yd, h->ldh, h->w, h->partial, h->ldp, h->arcnt,
                           h->krylov_m, j, h->fg, rtol, maxit, h->st));
    CK(seg_mul(h->nchunks, h->cbeg, h->cend, h->cseg, h->w, h->V + (size_t)(j + 1) * n, h->fg.scale, h->st,
               r32_out(h)));
    CK(cudaMemcpyAsync(h->hstat + j, h->fg.stat + j, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    return STOKES_OK;
  }
  TRY(seg_dots(h, h->V, n, nc, h->w, 0));
  CK(multiaxpy(h->nchunks, h->cbeg, h->cend, h->cseg, nc, h->V, n, h->hd, h->ldh, -1.0, h->w, h->st));
  CK(cudaMemcpyAsync(h->yd, h->hd, sizeof(double) * ni * h->ldh, cudaMemcpyDeviceToDevice, h->st));
  TRY(seg_dots(h, h->V, n, nc, h->w, 0));
  CK(multiaxpy(h->nchunks, h->cbeg, h->cend, h->cseg, nc, h->V, n, h->hd, h->ldh, -1.0, h->w, h->st));
  CK(multidot_partial(h->ndchunks, h->dbeg, h->dend, 1, h->w, 0, h->w, h->partial, h->ldp, h->st));
  CK(multidot_finish(ni, h->sd_beg, h->sd_end, 1, h->partial, h->ldp, h->yd + nc, h->ldh, 0, h->st));
  CK(fg_update(ni, h->krylov_m, j, h->fg, h->yd, h->hd, h->ldh, rtol, maxit, h->st));
  CK(seg_mul(h->nchunks, h->cbeg, h->cend, h->cseg, h->w, h->V + (size_t)(j + 1) * n, h->fg.scale, h->st,
             r32_out(h)));
  CK(cudaMemcpyAsync(h->hstat + j, h->fg.stat + j, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  return STOKES_OK;
}

// The Arnoldi step of column j as a CUDA graph (captured once per column,
// tolerance and iteration cap).
int iter_graph(stokes_handle* h, int j, double rtol, int maxit, cudaGraphExec_t* out) {
  auto key = std::make_tuple(j, rtol, maxit);
  auto it = h->iter_graphs.find(key);
  if (it != h->iter_graphs.end()) {
    *out = it->second;
    return STOKES_OK;
  }
  if (h->cycle_launches < 0) {
    h->led = Ledger();
    h->led.count = true;
    int rc0 = run_cycle(h, h->V, h->Z);
    h->led.count = false;
    TRY(rc0);
    h->cycle_launches = h->led.launches;
  }
  // kernel attributes are set at setup, so capture can start right away
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal));
  int rc = arnoldi_step(h, j, rtol, maxit);
  cudaError_t ec = cudaStreamEndCapture(h->st, &g);
  if (rc != STOKES_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  CK(ec);
  cudaGraphExec_t ge = nullptr;
  cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  CK(ei);
  h->iter_graphs[key] = ge;
  *out = ge;
  return STOKES_OK;
}

}  // namespace

extern "C" int stokes_fgmres_solve(stokes_handle* h, const double* b, double* x, double rtol, int32_t restart,
                                   int32_t maxit, stokes_solve_info* info) {
  if (!h || !b || !x || restart < 1 || restart > 1024 || maxit < 0 || !(rtol > 0))
    return fail(STOKES_ERR_INVALID_ARG, "fgmres arguments");
  if (!h->factored && h->precond == STOKES_PRECOND_DC) return fail(STOKES_ERR_STATE, "stokes_factor_patches must run first");
  const int m = restart;
  if (h->krylov_m != m) {
    h->krylov_m = 0;
    h->V = nullptr;
  }
  TRY(ensure_krylov(h, m));
  const int ni = h->ninst;
  const int64_t n = h->lv[0].n;
  Level& L0 = h->lv[0];
  TRY(join_in(h));
  CK(cudaMemsetAsync(h->fg.its, 0, sizeof(int) * ni, h->st));
  CK(cudaMemsetAsync(h->fg.err, 0, sizeof(int), h->st));
  // ||b|| per instance
  TRY(seg_dots(h, b, 0, 1, b, 0));
  CK(fg_start(ni, m, h->fg, h->hd, h->ldh, rtol, maxit, 1, h->st));
  int status = STOKES_OK;
  while (true) {
    // true residual r = b - K0 x into V_0, its norms, the start of a cycle
    CK((spmv<double, double, double, double, double>(L0.K, L0.K.v64, x, b, h->V, SPMV_RES, 0, 0, nullptr, h->st)));
    TRY(seg_dots(h, h->V, 0, 1, h->V, 0));
    CK(fg_start(ni, m, h->fg, h->hd, h->ldh, rtol, maxit, 0, h->st));
    CK(seg_mul(h->nchunks, h->cbeg, h->cend, h->cseg, h->V, h->V, h->fg.scale, h->st, r32_out(h)));
    CK(cudaMemcpyAsync(h->hstat + m, h->fg.stat + m, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (!h->hstat[m]) break;
    // Arnoldi steps: step j is queued before the flag of step j-1 is read,
    // so the device never waits for the host; a step queued after every
    // instance stopped works on zero vectors and changes nothing
    int last = -1;
    for (int j = 0; j < m; ++j) {
      cudaGraphExec_t ge;
      TRY(iter_graph(h, j, rtol, maxit, &ge));
      CK(cudaGraphLaunch(ge, h->st));
      h->launches += h->cycle_launches - (r32_input(h) ? 1 : 0) + (j + 1 <= kArMaxCols ? 5 : 11);
      CK(cudaEventRecord(h->ev_iter[j], h->st));
      last = j;
      if (j > 0) {
        CK(cudaEventSynchronize(h->ev_iter[j - 1]));
        if (!h->hstat[j - 1]) break;
      }
    }
    // x += Z y per instance
    CK(fg_solve(ni, m, h->fg, h->ldh, h->st));
    CK(multiaxpy(h->nchunks, h->cbeg, h->cend, h->cseg, m, h->Z, n, h->fg.y, h->ldh, 1.0, x, h->st));
    (void)last;
  }
  TRY(check_pipeline_errors(h));
  std::vector<int> its(ni), ferr(1);
  CK(cudaMemcpyAsync(its.data(), h->fg.its, sizeof(int) * ni, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(ferr.data(), h->fg.err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  // final true residuals
  CK((spmv<double, double, double, double, double>(L0.K, L0.K.v64, x, b, h->w, SPMV_RES, 0, 0, nullptr, h->st)));
  TRY(seg_dots(h, h->w, 0, 1, h->w, 0));
  std::vector<double> hbuf((size_t)ni * h->ldh), bn(ni);
  CK(cudaMemcpyAsync(hbuf.data(), h->hd, sizeof(double) * ni * h->ldh, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(bn.data(), h->fg.bnorm, sizeof(double) * ni, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (ferr[0]) return fail(STOKES_ERR_NAN, "non-finite value in the Krylov iteration");
  for (int s = 0; s < ni; ++s) {
    const double rr = bn[s] > 0 ? std::sqrt(hbuf[(size_t)s * h->ldh]) / bn[s] : 0.0;
    if (!std::isfinite(rr)) return fail(STOKES_ERR_NAN, "non-finite residual");
    const int st = rr <= rtol ? STOKES_OK : STOKES_NOT_CONVERGED;
    if (st != STOKES_OK) status = STOKES_NOT_CONVERGED;
    if (info) {
      info[s].iters = its[s];
      info[s].status = st;
      info[s].true_relres = rr;
    }
  }
  TRY(join_out(h));
  return status;
}

extern "C" int stokes_fgmres_solve_host(stokes_handle* h, const double* b_host, double* x_host, double rtol,
                                        int32_t restart, int32_t maxit, stokes_solve_info* info) {
  if (!h || !b_host || !x_host) return fail(STOKES_ERR_INVALID_ARG, "null argument");
  const int64_t n = h->lv[0].n;
  double *bd = nullptr, *xd = nullptr;
  CK(cudaMallocAsync(&bd, sizeof(double) * n, h->st));
  CK(cudaMallocAsync(&xd, sizeof(double) * n, h->st));
  CK(cudaMemcpyAsync(bd, b_host, sizeof(double) * n, cudaMemcpyHostToDevice, h->st));
  CK(cudaMemcpyAsync(xd, x_host, sizeof(double) * n, cudaMemcpyHostToDevice, h->st));
  int rc = stokes_fgmres_solve(h, bd, xd, rtol, restart, maxit, info);
  if (rc >= 0) {
    CK(cudaMemcpyAsync(x_host, xd, sizeof(double) * n, cudaMemcpyDeviceToHost, h->st));
  }
  cudaFreeAsync(bd, h->st);
  cudaFreeAsync(xd, h->st);
  CK(cudaStreamSynchronize(h->st));
  return rc;
}

// ------------------------------------------------------------- level ops
static int level_op_impl(stokes_handle* h, int32_t op, int32_t l, const double* x, const double* b, double* y);

template <typename T>
static int launch_one(stokes_handle* h, int which, int l) {
  Level& lv = h->lv[l];
  T* x = reinterpret_cast<T*>(lv.x);
  T* b = reinterpret_cast<T*>(lv.b);
  T* r = reinterpret_cast<T*>(lv.r);
  T* yp = reinterpret_cast<T*>(lv.yp);
  switch (which) {
    case STOKES_KERNEL_VANKA_APPLY: return L_apply<T, T>(h, lv, r, yp);
    case STOKES_KERNEL_SCATTER: return L_scatter<T>(h, lv, yp, x, lv.omega, 1);
    case STOKES_KERNEL_SPMV: return L_spmv<T, T, T, T, T>(h, lv.K, kval<T>(lv.K), x, b, r, SPMV_RES);
    default: {
      Level& l1 = h->lv[1];
      return L_spmv<double, T, double, T, double>(h, lv.K, lv.K.v64, x, reinterpret_cast<const double*>(lv.ta),
                                                  reinterpret_cast<T*>(l1.b), SPMV_SCALED_RES, h->eta_u, h->eta_p,
                                                  h->kind0);
    }
  }
}

extern "C" int stokes_time_kernel(stokes_handle* h, int32_t which, int32_t l, int32_t reps, double* avg_ms,
                                  double* bytes) {
  if (!h || l < 0 || l >= h->L || reps < 1 || which < 0 || which > 3) return fail(STOKES_ERR_INVALID_ARG, "time_kernel arguments");
  if ((which <= 1) && (!h->lv[l].has_patches || !h->factored)) return fail(STOKES_ERR_STATE, "level has no factored patches");
  if (which == 3 && (l != 0 || h->L < 2)) return fail(STOKES_ERR_INVALID_ARG, "DC residual is a level-0 kernel");
  const bool f32 = h->prec == STOKES_FP32;
  // byte count from the ledger
  h->led = Ledger();
  h->led.count = true;
  int rc = f32 ? launch_one<float>(h, which, l) : launch_one<double>(h, which, l);
  h->led.count = false;
  TRY(rc);
  if (bytes) *bytes = h->led.bytes;
  if (!h->flush) {
    h->flush_bytes = size_t(256) << 20;
    TRY(dalloc(h, reinterpret_cast<char**>(&h->flush), h->flush_bytes));
  }
  TRY(join_in(h));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double tot = 0.0;
  for (int k = 0; k < reps; ++k) {
    CK(l2_flush(h->flush, h->flush_bytes, h->st));
    CK(cudaEventRecord(e0, h->st));
    TRY(f32 ? launch_one<float>(h, which, l) : launch_one<double>(h, which, l));
    CK(cudaEventRecord(e1, h->st));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    tot += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (avg_ms) *avg_ms = tot / reps;
  return join_out(h);
}

extern "C" int stokes_inject_pipeline_error(stokes_handle* h, int32_t l) {
  if (!h || l < 0 || l >= h->L || !h->lv[l].has_patches) return fail(STOKES_ERR_INVALID_ARG, "level has no patches");
  const int v = 8;  // a flag value no pipeline sets (1, 2, 4 mark its own waits)
  CK(cudaMemcpyAsync(h->lv[l].pat.err, &v, sizeof(int), cudaMemcpyHostToDevice, h->st));
  CK(cudaStreamSynchronize(h->st));
  return STOKES_OK;
}

extern "C" int stokes_level_op(stokes_handle* h, int32_t op, int32_t l, const double* x, const double* b, double* y) {
  if (!h || l < 0 || l >= h->L || !y) return fail(STOKES_ERR_INVALID_ARG, "level_op arguments");
  TRY(join_in(h));
  TRY(level_op_impl(h, op, l, x, b, y));
  TRY(check_pipeline_errors(h));
  return join_out(h);
}

static int level_op_impl(stokes_handle* h, int32_t op, int32_t l, const double* x, const double* b, double* y) {
  Level& lv = h->lv[l];
  const bool f32 = h->prec == STOKES_FP32;
  auto in_cast = [&](int64_t n, const double* src, void* dst) -> int {
    if (f32) CK((cast_copy<double, float>(n, src, reinterpret_cast<float*>(dst), h->st)));
    else CK((cast_copy<double, double>(n, src, reinterpret_cast<double*>(dst), h->st)));
    return STOKES_OK;
  };
  auto out_cast = [&](int64_t n, const void* src, double* dst) -> int {
    if (f32) CK((cast_copy<float, double>(n, reinterpret_cast<const float*>(src), dst, h->st)));
    else CK((cast_copy<double, double>(n, reinterpret_cast<const double*>(src), dst, h->st)));
    return STOKES_OK;
  };
  switch (op) {
    case STOKES_OP_SPMV_F64:
      CK((spmv<double, double, double, double, double>(lv.K, lv.K.v64, x, x, y, SPMV_SET, 0, 0, nullptr, h->st)));
      return STOKES_OK;
    case STOKES_OP_SPMV:
    case STOKES_OP_RESIDUAL: {
      TRY(in_cast(lv.n, x, lv.ta));
      if (op == STOKES_OP_RESIDUAL) TRY(in_cast(lv.n, b, lv.b));
      const int mode = op == STOKES_OP_SPMV ? SPMV_SET : SPMV_RES;
      if (f32) CK((spmv<float, float, float, float, float>(lv.K, lv.K.v32, (float*)lv.ta, (float*)lv.b, (float*)lv.tb, mode, 0, 0, nullptr, h->st)));
      else CK((spmv<double, double, double, double, double>(lv.K, lv.K.v64, (double*)lv.ta, (double*)lv.b, (double*)lv.tb, mode, 0, 0, nullptr, h->st)));
      return out_cast(lv.n, lv.tb, y);
    }
    case STOKES_OP_RESTRICT:
    case STOKES_OP_PROLONG: {
      if (l + 1 >= h->L) return fail(STOKES_ERR_INVALID_ARG, "no coarser level");
      Level& lc = h->lv[l + 1];
      const bool restr = op == STOKES_OP_RESTRICT;
      const DevCSR& M = restr ? lv.R : lv.P;
      void* tin = restr ? lv.ta : lc.ta;
      void* tout = restr ? lc.tb : lv.tb;
      TRY(in_cast(restr ? lv.n : lc.n, x, tin));
      if (f32) CK((spmv<float, float, float, float, float>(M, M.v32, (float*)tin, (float*)nullptr, (float*)tout, SPMV_SET, 0, 0, nullptr, h->st)));
      else CK((spmv<double, double, double, double, double>(M, M.v64, (double*)tin, (double*)nullptr, (double*)tout, SPMV_SET, 0, 0, nullptr, h->st)));
      return out_cast(restr ? lc.n : lv.n, tout, y);
    }
    case STOKES_OP_VANKA:
    case STOKES_OP_RELAX: {
      if (!lv.has_patches && !(op == STOKES_OP_RELAX && lv.dlsc)) return fail(STOKES_ERR_INVALID_ARG, "level has no patches");
      if (!h->factored) return fail(STOKES_ERR_STATE, "stokes_factor_patches must run first");
      if (op == STOKES_OP_VANKA) {
        TRY(in_cast(lv.n, x, lv.ta));
        if (f32) {
          CK((vanka_apply<float, float>(lv.pat, (float*)lv.ta, (float*)lv.yp, h->st, &h->fj)));
          CK(vanka_scatter<float>(lv.pat, lv.n, (float*)lv.yp, (float*)lv.tb, 1.0, 0, nullptr, nullptr, nullptr, h->st));
        } else {
          CK((vanka_apply<double, double>(lv.pat, (double*)lv.ta, (double*)lv.yp, h->st, &h->fj)));
          CK(vanka_scatter<double>(lv.pat, lv.n, (double*)lv.yp, (double*)lv.tb, 1.0, 0, nullptr, nullptr, nullptr, h->st));
        }
        return out_cast(lv.n, lv.tb, y);
      }
      TRY(in_cast(lv.n, x, lv.tb));
      TRY(in_cast(lv.n, b, lv.ta));
      const int sweeps = lv.krylov ? lv.kmax : 1;
      if (f32) TRY(relax<float>(h, h->lv, l, (float*)lv.tb, (const float*)lv.ta, sweeps, false));
      else TRY(relax<double>(h, h->lv, l, (double*)lv.tb, (const double*)lv.ta, sweeps, false));
      return out_cast(lv.n, lv.tb, y);
    }
    case STOKES_OP_COARSE: {
      if (lv.coarse.nblocks == 0) return fail(STOKES_ERR_INVALID_ARG, "no coarsest blocks on this level");
      TRY(in_cast(lv.n, x, lv.ta));
      if (f32) CK(coarse_solve<float>(lv.coarse.nblocks, lv.coarse.boff, lv.coarse.bn, lv.coarse.koff, lv.coarse.Kinv, lv.coarse.max_n, (float*)lv.ta, (float*)lv.tb, h->st));
      else CK(coarse_solve<double>(lv.coarse.nblocks, lv.coarse.boff, lv.coarse.bn, lv.coarse.koff, lv.coarse.Kinv, lv.coarse.max_n, (double*)lv.ta, (double*)lv.tb, h->st));
      return out_cast(lv.n, lv.tb, y);
    }
    default:
      return fail(STOKES_ERR_INVALID_ARG, "unknown op");
  }
}
