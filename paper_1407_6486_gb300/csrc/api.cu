// api.cu -- C ABI, host-side set-up and the PFASST / SDC / multigrid schedule.
//
// Host set-up computes, in long double: Gauss-Lobatto nodes (eigenvalues of the
// Jacobi matrix of the (1,1) Jacobi polynomials, whose roots are those of P'_{s-1}),
// the integration matrix Q of Sec. 2.1 (moment equations of the interpolatory rule),
// the Lagrange time-interpolation matrix (barycentric form) and the exact inverse of
// the 3^d coarsest multigrid operator (sine eigen-decomposition).  The device work is
// the batched schedule of Sec. 2.2 - 2.4 on the kernels of kernels.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "pfasst_mg.h"
#include "pmg_internal.cuh"

using namespace pmg;

namespace {

thread_local std::string g_create_error;

// ----------------------------------------------------------------- nodes and Q

// Gauss-Lobatto nodes on [0,1]: endpoints plus the N-1 roots of P'_N (N = s-1), found
// by Sturm-sequence bisection on the symmetric tridiagonal Jacobi matrix of the
// Jacobi(1,1) polynomials (zero diagonal, off-diagonal sqrt(k(k+2)/((2k+1)(2k+3)))).
void gauss_lobatto(int s, long double *tau) {
  const int N = s - 1, m = N - 1;
  std::vector<long double> off(m > 1 ? m - 1 : 1);
  for (int k = 1; k <= m - 1; ++k) off[k - 1] = sqrtl((long double)k * (k + 2) / ((2.0L * k + 1) * (2.0L * k + 3)));
  auto count_below = [&](long double x) {
    int cnt = 0;
    long double d = 1.0L;
    for (int i = 0; i < m; ++i) {
      long double b2 = i > 0 ? off[i - 1] * off[i - 1] : 0.0L;
      d = (0.0L - x) - (i > 0 ? b2 / d : 0.0L);
      if (d == 0.0L) d = -1e-300L;
      if (d < 0) ++cnt;
    }
    return cnt;
  };
  tau[0] = 0.0L;
  tau[N] = 1.0L;
  for (int r = 0; r < m; ++r) {  // r-th smallest eigenvalue
    long double lo = -1.0L, hi = 1.0L;
    for (int it = 0; it < 200; ++it) {
      long double mid = 0.5L * (lo + hi);
      if (count_below(mid) > r) hi = mid; else lo = mid;
    }
    tau[r + 1] = (0.5L * (lo + hi) + 1.0L) / 2.0L;
  }
}

// Q[m][j]: weights of the interpolatory rule for the integral over [0, tau_m]:
// sum_j Q[m][j] tau_j^k = tau_m^{k+1}/(k+1), k = 0..s-1 (Gaussian elimination).
// Node positions on [0,1]: family 0 Gauss-Lobatto, family 1 uniform m/(s-1) (the
// paper's second- and fourth-order methods, Sec. 3).
void node_positions(int s, int family, long double *tau) {
  if (family == 0) {
    gauss_lobatto(s, tau);
    return;
  }
  for (int m = 0; m < s; ++m) tau[m] = (long double)m / (long double)(s - 1);
}

// Integration matrix from the moment equations of the interpolatory rule: row m holds
// the weights that integrate polynomials of degree < (number of rule nodes) exactly
// over [0, tau_m].  Family 0 interpolates through all s nodes; family 1 through
// tau_1..tau_{s-1} only (the rule without the left endpoint; column 0 is zero).
void integration_matrix(int s, const long double *tau, long double Q[kMaxNodes][kMaxNodes], int family = 0) {
  const int j0 = family == 1 ? 1 : 0, nr = s - j0;  // first rule node, rule size
  for (int m = 0; m < s; ++m) {
    long double A[kMaxNodes][kMaxNodes + 1];
    for (int k = 0; k < nr; ++k) {
      for (int j = 0; j < nr; ++j) A[k][j] = powl(tau[j0 + j], k);
      A[k][nr] = powl(tau[m], k + 1) / (k + 1);
    }
    for (int col = 0; col < nr; ++col) {
      int piv = col;
      for (int r = col + 1; r < nr; ++r)
        if (fabsl(A[r][col]) > fabsl(A[piv][col])) piv = r;
      for (int q = 0; q <= nr; ++q) { long double t = A[col][q]; A[col][q] = A[piv][q]; A[piv][q] = t; }
      for (int r = 0; r < nr; ++r) {
        if (r == col) continue;
        long double f = A[r][col] / A[col][col];
        for (int q = col; q <= nr; ++q) A[r][q] -= f * A[col][q];
      }
    }
    for (int j = 0; j < j0; ++j) Q[m][j] = 0.0L;
    for (int j = 0; j < nr; ++j) Q[m][j0 + j] = A[j][nr] / A[j][j];
  }
}

// Lagrange weights of the coarse nodes tc at the point t (barycentric form)
void lagrange_row(int sc, const long double *tc, long double t, double *row) {
  for (int j = 0; j < sc; ++j)
    if (fabsl(t - tc[j]) < 1e-15L) {
      for (int q = 0; q < sc; ++q) row[q] = q == j ? 1.0 : 0.0;
      return;
    }
  long double lam[kMaxNodes], den = 0.0L;
  for (int j = 0; j < sc; ++j) {
    lam[j] = 1.0L;
    for (int i = 0; i < sc; ++i)
      if (i != j) lam[j] /= (tc[j] - tc[i]);
    den += lam[j] / (t - tc[j]);
  }
  for (int j = 0; j < sc; ++j) row[j] = (double)((lam[j] / (t - tc[j])) / den);
}

// exact inverse of (I - c Lap_h) on the 3^dim grid (h = 1/4) from the sine
// eigenvectors v_k(i) = sqrt(1/2) sin(k pi (i+1)/4) of the 1D operator
void coarsest_inverse(int dim, double c, std::vector<double> &out) {
  const int N3 = dim == 1 ? 3 : (dim == 2 ? 9 : 27);
  out.assign((size_t)N3 * N3, 0.0);
  const long double pi = 3.14159265358979323846264338327950288L;
  long double v[3][3], mu[3];
  for (int k = 0; k < 3; ++k) {
    mu[k] = (2.0L * cosl((k + 1) * pi / 4.0L) - 2.0L) * 16.0L;
    for (int i = 0; i < 3; ++i) v[k][i] = sqrtl(0.5L) * sinl((k + 1) * pi * (i + 1) / 4.0L);
  }
  auto decode = [&](int p, int *ix) { ix[0] = p % 3; ix[1] = (p / 3) % 3; ix[2] = p / 9; };
  for (int p = 0; p < N3; ++p)
    for (int q = 0; q < N3; ++q) {
      int pi3[3], qi3[3];
      decode(p, pi3);
      decode(q, qi3);
      long double acc = 0.0L;
      for (int kk = 0; kk < N3; ++kk) {
        int ks[3];
        decode(kk, ks);
        long double lam = 1.0L, prod = 1.0L;
        for (int a = 0; a < dim; ++a) {
          lam -= (long double)c * mu[ks[a]];
          prod *= v[ks[a]][pi3[a]] * v[ks[a]][qi3[a]];
        }
        acc += prod / lam;
      }
      out[(size_t)p * N3 + q] = (double)acc;
    }
}

bool is_pow2_minus1(int n) { return n >= 3 && ((n + 1) & n) == 0; }

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// ----------------------------------------------------------------- hierarchy

// Smoother choice of one level: the fused red-black z-marching sweep (fused = 1; param =
// z chunk, 0 = default), its TMA-staged variant (fused = 2, FP32), or the
// one-point-per-thread kernels (fused = 0; param = threads per block).
struct Tune {
  int fused = 0;
  int param = 256;    // per-point kernels: threads per block; fused sweep: z chunk (0 = default)
  int threads = 256;  // fused sweep: threads per CTA
};

struct Hier {
  int L = 0;
  Grid lev[kMaxLevels];
  void *e[kMaxLevels] = {}, *e2[kMaxLevels] = {}, *f[kMaxLevels] = {};
  Prec pr = F64;
  size_t tsize = 8;
  int batch = 1;                  // grids per level the buffers hold
  Tune tune[kMaxLevels][2];       // [level][0: wide batches, 1: narrow (a single grid)]
  int tail = -1;                  // first level of the one-launch V-cycle bottom (-1: none)
  VTailDesc td;                   // its shared-memory plan
  unsigned *count = nullptr;      // grid-barrier word of the persistent single-grid V-cycle
  // wide tuning for batches of a few grids or more (slice groups), narrow for single grids
  const Tune &tune_for(int l, int B) const { return tune[l][(2 * B >= batch || B >= 4) ? 0 : 1]; }
};

int mg_levels(int n) {
  int L = 1;
  while (n > 3) { n = (n - 1) / 2; ++L; }
  return L;
}

// memory plan: a list of (pointer slot, bytes) carved from one block
struct Plan {
  std::vector<std::pair<void **, size_t>> items;
  size_t total = 0;
  void add(void **slot, size_t bytes) { items.push_back({slot, bytes}); total += align256(bytes); }
  void carve(char *base) {
    size_t o = 0;
    for (auto &it : items) { *it.first = base + o; o += align256(it.second); }
  }
};

}  // namespace

// ----------------------------------------------------------------- handle

constexpr int kMaxGroups = 8;  // slice groups of the pipelined PFASST iteration

// learned correction network deployed in the V-cycles of a handle: on every level
// with on[l], the second pre-smoothing sweep is replaced by e += net(D^-1 r)
struct NetDeploy {
  void *mem = nullptr;  // parameters + scratch, one cudaMalloc
  float *prm = nullptr;
  NetScratch s;
  int chunk = 1;        // grids per correction launch (bounds the scratch)
  bool on[kMaxLevels] = {};
};

// the device-side PFASST iteration loop: the host writes max_iter and tol, the check
// kernel at the end of every iteration counts k and keeps the residual (max over slices)
struct LoopCtl {
  int max_iter;
  int k;
  double tol;
  unsigned long long res_bits;
};

struct pmg_ctx {
  int dim = 0, nf = 0, nc = 0, sf = 0, sc = 0, P = 0, nlevels = 1;
  int order = 2;           // Laplacian stencil of the fine level (coarser levels: 2)
  int famf = 0, famc = 0;  // node families (0 Gauss-Lobatto, 1 uniform)
  double nu = 0, dt = 0;
  pmg_options opt{};
  pmg_options opt_c{};     // options of the coarse PFASST levels' sub-step solves (coarse_vcycles)
  cudaStream_t stream = nullptr;
  Grid gf{}, gc{}, gd{};
  long double tauf[kMaxNodes] = {}, tauc[kMaxNodes] = {};
  SFCoef sff{}, sfc{};
  ResCoef resf{};
  FASCoef fas{};
  InterpCoef interp{};
  double cf_sub[kMaxNodes] = {}, cc_sub[kMaxNodes] = {};  // c_m = dt_m nu per sub-step
  // device state
  double *Uf = nullptr, *Ff = nullptr, *qf = nullptr, *u0 = nullptr, *dense = nullptr;
  double *Uc = nullptr, *Fc = nullptr, *qc = nullptr, *tau = nullptr, *Uc0 = nullptr;
  // time-interpolated coarse correction [slice][fine node][coarse grid], MG precision
  void *dU = nullptr;
  // level 2 of a three-level hierarchy: grid (n-3)/4, s2 nodes of family fam2
  int s2 = 0, fam2 = 0;
  Grid g2{};
  long double tau2n[kMaxNodes] = {};
  SFCoef sf2c{};
  FASCoef fas2{};        // restriction level 1 -> 2
  InterpCoef interp2{};  // correction level 2 -> 1
  double c2_sub[kMaxNodes] = {};
  double *U2 = nullptr, *F2 = nullptr, *q2 = nullptr, *tau2 = nullptr, *U20 = nullptr;
  void *dU2 = nullptr;   // [slice][level-1 node][level-2 grid], MG precision
  Hier H;
  void *minv = nullptr;  // (sf-1) + (sc-1) + (s2-1) slots of N3*N3 in MG precision
  int n3 = 3;
  unsigned long long *red = nullptr;  // [3P]: rnorm, bnorm, colloc residual
  int *active = nullptr;
  unsigned long long *hred = nullptr;  // pinned
  LoopCtl *ctl = nullptr;               // device-side iteration loop: limits and results
  LoopCtl *hctl = nullptr;              // pinned
  bool in_loop = false;                 // capturing the body of the device-side loop
  int *hactive = nullptr;              // pinned
  void *ws = nullptr;
  bool ws_owned = false;
  bool predicted = false;
  bool spread_state = false;  // every slice holds the spread initial value (nothing has run since)
  bool q_valid = false;  // F-free mode: qf holds the right-hand sides of the current U_f
  long long launches = 0;
  Profiler prof;
  // CUDA graphs of the predictor and of one PFASST iteration (fixed V-cycle counts)
  struct Captured {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
    bool with_prof = false;
    long long prof_min = 0;
    std::vector<ProfRec> recs;
  } g_pred, g_pred_spread, g_iter, g_loop;
  cudaStream_t cap_stream = nullptr;
  // uneven batch: one single-level solver per problem, run as branches of one graph
  std::vector<pmg_ctx *> kids;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t bexec = nullptr;
  int bsweeps = -1;
  long long bkernels = 0;
  NetDeploy *net = nullptr;
  // slice-group pipeline of a PFASST iteration: the coarse chain of group g runs on
  // s_chain (high priority, own multigrid scratch Hc) while the fine sweeps of later
  // groups run on the main stream; interpolation, send-forward and residual of group g
  // follow on s_post
  int groups = 1;
  Hier Hc;
  Hier *mgH = nullptr;  // hierarchy the multigrid schedule uses (null: H)
  cudaStream_t s_chain = nullptr, s_post = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_chain_end = nullptr, ev_post_end = nullptr;
  cudaEvent_t ev_fas[kMaxGroups] = {}, ev_chain[kMaxGroups] = {};
  std::string err;

  Launch L() { return Launch{stream, &launches, &prof}; }
  const void *minv_slot(int slot) const { return (const char *)minv + (size_t)slot * n3 * n3 * H.tsize; }
};

namespace {

int fail(pmg_ctx *h, int code, const std::string &msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return code;
}

#define PMG_CUDA(h, expr)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(h, PMG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));    \
  } while (0)

#define PMG_RET(expr)            \
  do {                           \
    int r_ = (expr);             \
    if (r_ != PMG_OK) return r_; \
  } while (0)

int validate(const pmg_grid *grid, const pmg_nodes_desc *fn, const pmg_levels *lv, int slices,
             const pmg_options *o, std::string &why) {
  if (!grid || !fn || !lv) { why = "null description"; return PMG_ERR_INVALID_ARG; }
  if (grid->dim < 1 || grid->dim > 3) { why = "dim must be 1, 2 or 3"; return PMG_ERR_INVALID_ARG; }
  if (!is_pow2_minus1(grid->n) || grid->n > 1023) { why = "n must be 2^p - 1 in [3, 1023]"; return PMG_ERR_INVALID_ARG; }
  if (grid->order != 0 && grid->order != 2 && grid->order != 4) { why = "order must be 0, 2 or 4"; return PMG_ERR_INVALID_ARG; }
  if (grid->order == 4 && grid->n < 7) { why = "the fourth-order stencil needs n >= 7"; return PMG_ERR_INVALID_ARG; }
  if (fn->family != 0 && fn->family != 1) { why = "node family must be 0 (Gauss-Lobatto) or 1 (uniform)"; return PMG_ERR_UNSUPPORTED; }
  if (fn->count < 2 || fn->count > kMaxNodes) { why = "fine node count must be in [2, 9]"; return PMG_ERR_INVALID_ARG; }
  if (lv->nlevels < 1 || lv->nlevels > 3) { why = "nlevels must be 1, 2 or 3"; return PMG_ERR_INVALID_ARG; }
  if (lv->nlevels >= 2) {
    if (lv->coarse_nodes.family != 0 && lv->coarse_nodes.family != 1) {
      why = "coarse node family must be 0 (Gauss-Lobatto) or 1 (uniform)";
      return PMG_ERR_UNSUPPORTED;
    }
    if (lv->coarse_nodes.count < 2 || lv->coarse_nodes.count > fn->count) { why = "bad coarse node count"; return PMG_ERR_INVALID_ARG; }
    if (grid->n < 7) { why = "two levels need n >= 7"; return PMG_ERR_INVALID_ARG; }
  }
  if (lv->nlevels == 3) {
    if (lv->coarsest_nodes.family != 0 && lv->coarsest_nodes.family != 1) {
      why = "coarsest node family must be 0 (Gauss-Lobatto) or 1 (uniform)";
      return PMG_ERR_UNSUPPORTED;
    }
    if (lv->coarsest_nodes.count < 2 || lv->coarsest_nodes.count > lv->coarse_nodes.count) {
      why = "bad coarsest node count";
      return PMG_ERR_INVALID_ARG;
    }
    if (grid->n < 15) { why = "three levels need n >= 15"; return PMG_ERR_INVALID_ARG; }
  }
  if (slices < 1 || slices > 4096) { why = "slices must be in [1, 4096]"; return PMG_ERR_INVALID_ARG; }
  if (o) {
    if (o->smoother != PMG_SMOOTHER_JACOBI && o->smoother != PMG_SMOOTHER_RBGS) { why = "bad smoother"; return PMG_ERR_INVALID_ARG; }
    if (o->nu1 < 0 || o->nu2 < 0 || o->nu1 + o->nu2 == 0 || o->nu1 > 16 || o->nu2 > 16) { why = "bad nu1/nu2"; return PMG_ERR_INVALID_ARG; }
    if (o->vcycles < 0 || o->vcycles > 1000) { why = "bad vcycles"; return PMG_ERR_INVALID_ARG; }
    if (o->coarse_vcycles < -1 || o->coarse_vcycles > 1000) { why = "bad coarse_vcycles"; return PMG_ERR_INVALID_ARG; }
    if (o->single_grid_vcycle != 0 && o->single_grid_vcycle != 1) {
      why = "single_grid_vcycle must be 0 or 1";
      return PMG_ERR_INVALID_ARG;
    }
    if ((o->vcycles == 0 || o->coarse_vcycles == 0) && (o->mg_maxcycles < 1 || !(o->mg_tol > 0))) {
      why = "bad full-solve settings";
      return PMG_ERR_INVALID_ARG;
    }
    if (o->precision != PMG_PREC_FP64 && o->precision != PMG_PREC_MIXED) { why = "bad precision"; return PMG_ERR_INVALID_ARG; }
    if (o->interp_order != 2 && o->interp_order != 4) { why = "interp_order must be 2 or 4"; return PMG_ERR_INVALID_ARG; }
    if (o->vcycle_tail < -1 || o->vcycle_tail > 1) { why = "vcycle_tail must be -1, 0 or 1"; return PMG_ERR_INVALID_ARG; }
    if (o->slice_groups < 0 || o->slice_groups > kMaxGroups) {
      why = "slice_groups must be 0 (automatic) .. 8";
      return PMG_ERR_INVALID_ARG;
    }
    if (!(o->omega > 0) || o->omega > 2) { why = "omega must be in (0, 2]"; return PMG_ERR_INVALID_ARG; }
  }
  return PMG_OK;
}

// the z-marching tiled kernels pay off on large batched 3D grids; small or batch-1
// grids (coarse levels, the serial coarse chain) keep the one-thread-per-point kernels
bool tiled3d(const Grid &g, int B) {
  return g.dim == 3 && g.order != 4 && g.n >= kTiled3dMinN && (long long)g.n * g.n * g.n * B >= (1LL << 24);
}

int grid_order(const pmg_grid *grid) { return grid->order == 4 ? 4 : 2; }

// multigrid hierarchy for `batch` grids of size n (levels n, (n-1)/2, ..., 3)
// buffers of levels >= first (the levels a V-cycle from `first` touches); order0 is the
// stencil of the finest grid (the coarser grids are rediscretised with 2nd order)
void plan_hier(Plan &pl, Hier &H, int dim, int n, int batch, Prec pr, int smoother, int first = 0,
               int order0 = 2) {
  H.L = mg_levels(n);
  H.pr = pr;
  H.tsize = pr == F64 ? 8 : 4;
  H.batch = batch;
  int nl = n;
  for (int l = 0; l < H.L; ++l) {
    H.lev[l] = make_grid(dim, nl, l == 0 ? order0 : 2);
    for (int cls = 0; cls < 2; ++cls) {  // default choice; the autotuner may replace it
      Tune &t = H.tune[l][cls];
      t.fused = smoother == PMG_SMOOTHER_RBGS && tiled3d(H.lev[l], cls == 0 ? batch : 1);
      t.param = t.fused ? 0 : 256;
    }
    size_t bytes = (size_t)H.lev[l].slab * batch * H.tsize;
    if (l >= first) {
      pl.add(&H.e[l], bytes);
      pl.add(&H.f[l], bytes);
      // second correction buffer: Jacobi ping-pong, the out-of-place fused 3D sweep, or
      // the residual scratch of the persistent single-grid V-cycle (2D)
      if (smoother == PMG_SMOOTHER_JACOBI || dim >= 2) pl.add(&H.e2[l], bytes);
    }
    nl = (nl - 1) / 2;
  }
  pl.add((void **)&H.count, 256);
  // the finest level from which the rest of the V-cycle fits one CTA's shared memory
  // (at least two levels, so that the tail replaces several launches)
  H.tail = -1;
  for (int l = H.lev[0].order == 4 ? 1 : 0; l + 1 < H.L; ++l) {  // (the tail runs the 2nd-order stencil)
    VTailDesc d;
    if (vtail_plan(dim, H.lev[l].n, H.L - l, smoother == PMG_SMOOTHER_JACOBI ? 0 : 1, H.tsize, d) <= kVTailMaxSmem) {
      H.tail = l;
      H.td = d;
      break;
    }
  }
}

// coarsest-grid inverses: one per sub-step of every level, finest level first
int minv_slots(const pmg_ctx *h) {
  return (h->sf - 1) + (h->nlevels >= 2 ? h->sc - 1 : 0) + (h->nlevels == 3 ? h->s2 - 1 : 0);
}

void plan_ctx(Plan &pl, pmg_ctx *h) {
  const size_t sf = (size_t)h->gf.slab * 8;
  pl.add((void **)&h->Uf, sf * h->P * h->sf);
  // the fine F = A U is stored only for full solves (tolerance mode); with fixed V-cycle
  // counts the end-of-iteration pass and the FAS restriction evaluate it from U
  if (h->opt.vcycles == 0) pl.add((void **)&h->Ff, sf * h->P * h->sf);
  pl.add((void **)&h->qf, sf * h->P * (h->sf - 1));
  pl.add((void **)&h->u0, sf);
  pl.add((void **)&h->dense, sf);
  if (h->nlevels >= 2) {
    const size_t sc = (size_t)h->gc.slab * 8;
    pl.add((void **)&h->Uc, sc * h->P * h->sc);
    pl.add((void **)&h->Fc, sc * h->P * h->sc);
    pl.add((void **)&h->tau, sc * h->P * h->sc);
    pl.add((void **)&h->Uc0, sc * h->P * h->sc);
    pl.add((void **)&h->qc, sc * h->P * (h->sc - 1));
  }
  if (h->nlevels == 3) {
    const size_t s2 = (size_t)h->g2.slab * 8;
    pl.add((void **)&h->U2, s2 * h->P * h->s2);
    pl.add((void **)&h->F2, s2 * h->P * h->s2);
    pl.add((void **)&h->tau2, s2 * h->P * h->s2);
    pl.add((void **)&h->U20, s2 * h->P * h->s2);
    pl.add((void **)&h->q2, s2 * h->P * (h->s2 - 1));
  }
  const Prec pr = h->opt.precision == PMG_PREC_MIXED ? F32 : F64;
  plan_hier(pl, h->H, h->dim, h->nf, h->P, pr, h->opt.smoother, 0, h->order);
  if (h->groups > 1) plan_hier(pl, h->Hc, h->dim, h->nf, 1, pr, h->opt.smoother, 1, h->order);  // coarse chain scratch
  if (h->nlevels >= 2) pl.add(&h->dU, (size_t)h->gc.slab * h->P * h->sf * h->H.tsize);
  if (h->nlevels == 3) pl.add(&h->dU2, (size_t)h->g2.slab * h->P * h->sc * h->H.tsize);
  const int slots = minv_slots(h);
  pl.add(&h->minv, (size_t)slots * h->n3 * h->n3 * h->H.tsize);
  pl.add((void **)&h->red, sizeof(unsigned long long) * 3 * h->P);
  pl.add((void **)&h->active, sizeof(int) * h->P);
  pl.add((void **)&h->ctl, sizeof(LoopCtl));
}

// ----------------------------------------------------------------- multigrid schedule

struct MGCtx {
  Launch L;
  Hier *H;
  const pmg_options *o;
  unsigned long long *red;  // [2 * batch] norms (full-solve mode)
  int *active;              // [batch]
  unsigned long long *hred;
  int *hactive;
  pmg_ctx *h;               // for error messages (may be null)
  cudaStream_t stream;
  const NetDeploy *net = nullptr;  // learned correction (may be null)
};

// one smoothing sweep on level l with the smoother variant t; with the fused 3D
// red-black kernel and a non-null u_upd the sweep's result is added to u_upd (stride
// su) instead of being stored
int smooth_with(MGCtx &M, const Tune &t, int l, int B, double c, void *&cur, bool first, double *u_upd = nullptr,
                long long su = 0) {
  Hier &H = *M.H;
  const pmg_options &o = *M.o;
  if (o.smoother == PMG_SMOOTHER_JACOBI) {
    void *out = cur == H.e[l] ? H.e2[l] : H.e[l];
    PMG_CUDA(M.h, k_smooth_jacobi(M.L, H.lev[l], c, o.omega, H.pr, cur, out, H.f[l], B, first, t.param));
    cur = out;
  } else if (t.fused >= 2) {
    void *out = cur == H.e[l] ? H.e2[l] : H.e[l];
    PMG_CUDA(M.h, k_rbgs_sweep3d_tma(M.L, H.lev[l], c, o.omega, cur, out, H.f[l], u_upd, su, B, first,
                                     u_upd != nullptr, t.param, t.fused == 3));
    cur = out;
  } else if (t.fused) {
    void *out = cur == H.e[l] ? H.e2[l] : H.e[l];
    PMG_CUDA(M.h, k_rbgs_sweep3d(M.L, H.lev[l], c, o.omega, H.pr, cur, out, H.f[l], u_upd, su, B, first,
                                 u_upd != nullptr, t.param, t.threads));
    cur = out;
  } else {  // red, black (and a third colour for the fourth-order stencil)
    for (int colour = 0; colour < (H.lev[l].order == 4 ? 3 : 2); ++colour)
      PMG_CUDA(M.h, k_smooth_rbgs(M.L, H.lev[l], c, o.omega, H.pr, cur, H.f[l], B, colour, first && colour == 0,
                                  t.param));
  }
  return PMG_OK;
}

int smooth(MGCtx &M, int l, int B, double c, void *&cur, bool first, double *u_upd = nullptr, long long su = 0) {
  return smooth_with(M, M.H->tune_for(l, B), l, B, c, cur, first, u_upd, su);
}

// learned correction on level l: e += net(D^-1 (f - (I - c Lap) e)), in chunks of
// net->chunk grids so that the activations fit the scratch
int net_correct(MGCtx &M, int l, int B, double c, void *e) {
  Hier &H = *M.H;
  const Grid &g = H.lev[l];
  const size_t gb = (size_t)g.slab * H.tsize;
  for (int b0 = 0; b0 < B; b0 += M.net->chunk) {
    const int nb = B - b0 < M.net->chunk ? B - b0 : M.net->chunk;
    PMG_CUDA(M.h, k_net_correct(M.L, g, c, H.pr, (char *)e + b0 * gb, (const char *)H.f[l] + b0 * gb, nb,
                                M.net->prm, M.net->s));
  }
  return PMG_OK;
}

// one V(nu1,nu2)-cycle for (I - c Lap) e = f[l0] on levels l0..L-1, starting from
// e = 0 (e_init null) or from e_init (a buffer of level l0); *eout = result.
// If u_upd is non-null and the last post-smoothing sweep on level l0 can be fused
// with the update, u_upd += e is done there and *fused is set (then *eout is stale).
int vcycle(MGCtx &M, int l0, int B, double c, const void *minv, void *e_init, void **eout,
           double *u_upd = nullptr, long long su = 0, bool *fused = nullptr) {
  Hier &H = *M.H;
  const pmg_options &o = *M.o;
  void *cur[kMaxLevels];
  if (fused) *fused = false;
  // levels from lb down run in one launch for single grids (one CTA per grid: wide
  // batches keep the per-level kernels, which spread each level over many CTAs), unless
  // a learned correction acts there
  int lb = H.L;
  // automatic (-1): one launch in 1D and for red-black Gauss-Seidel, where it measured
  // faster than the per-level launches (1D, 3D and the uneven batch); per level for
  // weighted Jacobi in 2D and 3D (slower with the tail on the 2D workload)
  const int dim = H.lev[0].dim;
  const bool tail_on = o.vcycle_tail == 1 ||
                       (o.vcycle_tail == -1 && (dim == 1 || o.smoother == PMG_SMOOTHER_RBGS));
  if (tail_on && H.tail >= l0 && B <= 2) {
    lb = H.tail;
    if (M.net)
      for (int l = H.tail; l < H.L; ++l)
        if (M.net->on[l]) lb = H.L;
  }
  for (int l = l0; l < H.L - 1 && l < lb; ++l) {
    const bool zero = l > l0 || e_init == nullptr;
    cur[l] = zero ? H.e[l] : e_init;
    if (o.nu1 == 0 && zero) PMG_CUDA(M.h, k_zero(M.L, H.lev[l], H.pr, cur[l], B));
    for (int s = 0; s < o.nu1; ++s) {
      if (s == 1 && M.net && M.net->on[l]) PMG_RET(net_correct(M, l, B, c, cur[l]));
      else PMG_RET(smooth(M, l, B, c, cur[l], zero && s == 0));
    }
    if (tiled3d(H.lev[l], B))
      PMG_CUDA(M.h, resrestrict_tma_supported(H.lev[l], H.pr)
                        ? k_resrestrict3d_tma(M.L, H.lev[l], H.lev[l + 1], c, cur[l], H.f[l], H.f[l + 1], B)
                        : k_resrestrict3d(M.L, H.lev[l], H.lev[l + 1], c, H.pr, cur[l], H.f[l], H.f[l + 1], B));
    else
      PMG_CUDA(M.h, k_residual_restrict(M.L, H.lev[l], H.lev[l + 1], c, H.pr, cur[l], H.f[l], H.f[l + 1], B));
  }
  int ltop = H.L - 1;
  if (lb < H.L) {
    VTailDesc d = H.td;
    d.c = c;
    d.omega = o.omega;
    d.smoother = o.smoother == PMG_SMOOTHER_JACOBI ? 0 : 1;
    d.nu1 = o.nu1;
    d.nu2 = o.nu2;
    const void *ein = (lb == l0 && e_init) ? e_init : nullptr;
    PMG_CUDA(M.h, k_vcycle_tail(M.L, H.lev[lb], d, H.pr, minv, H.f[lb], ein, H.e[lb], B));
    cur[lb] = H.e[lb];
    ltop = lb;
  } else {
    PMG_CUDA(M.h, k_coarse_solve(M.L, H.lev[ltop], H.pr, minv, H.f[ltop], H.e[ltop], B));
    cur[ltop] = H.e[ltop];
  }
  for (int l = ltop - 1; l >= l0; --l) {
    if (H.lev[l].dim == 3 && H.lev[l].n >= 15)
      PMG_CUDA(M.h, k_prolong3d(M.L, H.lev[l], H.lev[l + 1], H.pr, cur[l + 1], cur[l], B));
    else
      PMG_CUDA(M.h, k_prolong_add(M.L, H.lev[l], H.lev[l + 1], H.pr, cur[l + 1], cur[l], B));
    for (int s = 0; s < o.nu2; ++s) {
      const bool last = l == l0 && s == o.nu2 - 1;
      const bool fuse = last && u_upd && o.smoother == PMG_SMOOTHER_RBGS && H.tune_for(l, B).fused;
      PMG_RET(smooth(M, l, B, c, cur[l], false, fuse ? u_upd : nullptr, su));
      if (fuse && fused) *fused = true;
    }
  }
  *eout = cur[l0];
  return PMG_OK;
}

// Solve (I - c Lap) u1 = um + qm for B grids on hierarchy level l0 (fixed V-cycles or
// full solve with the tolerance / stall rule).  *cycles = max cycles over the batch.
int solve_substep(MGCtx &M, int l0, int B, double c, const void *minv, const double *um, long long sum,
                  const double *qm, long long sq, double *u1, long long s1, int *cycles, bool pointwise = false) {
  Hier &H = *M.H;
  const pmg_options &o = *M.o;
  const Grid &g = H.lev[l0];
  if (o.vcycles > 0) {
    // one residual of the sub-step equation, then the V-cycles iterate on the
    // correction equation (I - c Lap) e = r from e = 0, then u1 += e: equal in exact
    // arithmetic to vcycles V-cycles applied to u1 itself
    void *e = nullptr;
    bool fused = false;
    if (pointwise)  // u_m + q_m already is the residual (see SFCoef)
      PMG_CUDA(M.h, k_resid_pt(M.L, g, H.pr, um, sum, qm, sq, H.f[l0], B));
    else
      PMG_CUDA(M.h, k_residual0(M.L, g, c, H.pr, um, sum, qm, sq, u1, s1, H.f[l0], B, nullptr, nullptr));
    // a single grid (the serial coarse chain): every V-cycle and the update in one
    // persistent launch, unless a learned correction acts on one of the levels
    bool net_here = false;
    for (int l = l0; M.net && l < H.L; ++l) net_here = net_here || M.net->on[l];
    if (B == 1 && o.single_grid_vcycle && !net_here &&
        vcycle_coop_supported(g, H.L - l0, o.smoother == PMG_SMOOTHER_RBGS, o.nu1)) {
      void *ev[kMaxLevels], *fv[kMaxLevels], *rv[kMaxLevels];
      for (int l = l0; l < H.L; ++l) {
        ev[l - l0] = H.e[l];
        fv[l - l0] = H.f[l];
        rv[l - l0] = H.e2[l];  // free during a red-black V-cycle: the residual scratch
      }
      PMG_CUDA(M.h, k_vcycle_coop(M.L, &H.lev[l0], H.L - l0, H.pr, c, o.omega, o.nu1, o.nu2, o.vcycles, ev, fv, rv,
                                  minv, u1, H.count));
      if (cycles) *cycles = o.vcycles;
      return PMG_OK;
    }
    for (int v = 0; v < o.vcycles; ++v) {
      const bool last = v == o.vcycles - 1;
      PMG_RET(vcycle(M, l0, B, c, minv, e, &e, last ? u1 : nullptr, s1, last ? &fused : nullptr));
    }
    if (!fused) PMG_CUDA(M.h, k_update_u(M.L, g, H.pr, u1, s1, e, B, nullptr));
    if (cycles) *cycles = o.vcycles;
    return PMG_OK;
  }
  // full solve (host-driven, per-grid activity mask)
  std::vector<double> r(B), bn(B);
  std::vector<int> done(B), cyc(B, 0);
  auto norms = [&](std::vector<double> &rr, std::vector<double> *bb) -> int {
    PMG_CUDA(M.h, cudaMemsetAsync(M.red, 0, sizeof(unsigned long long) * 2 * B, M.stream));
    PMG_CUDA(M.h, k_residual0(M.L, g, c, H.pr, um, sum, qm, sq, u1, s1, H.f[l0], B, M.red, M.red + B));
    PMG_CUDA(M.h, cudaMemcpyAsync(M.hred, M.red, sizeof(unsigned long long) * 2 * B, cudaMemcpyDeviceToHost, M.stream));
    PMG_CUDA(M.h, cudaStreamSynchronize(M.stream));
    for (int p = 0; p < B; ++p) {
      unsigned long long rv = M.hred[p], bv = M.hred[B + p];
      double rd, bd;
      std::memcpy(&rd, &rv, 8);
      std::memcpy(&bd, &bv, 8);
      if (std::isnan(rd) || std::isinf(rd)) return fail(M.h, PMG_ERR_DIVERGED, "NaN/Inf in a sub-step residual");
      rr[p] = rd;
      if (bb) (*bb)[p] = bd < 1.0 ? 1.0 : bd;
    }
    return PMG_OK;
  };
  PMG_RET(norms(r, &bn));
  int left = 0;
  for (int p = 0; p < B; ++p) {
    done[p] = !(r[p] > o.mg_tol * bn[p]);
    left += !done[p];
  }
  std::vector<double> rn(B);
  for (int it = 0; left > 0 && it < o.mg_maxcycles; ++it) {
    for (int p = 0; p < B; ++p) M.hactive[p] = !done[p];
    PMG_CUDA(M.h, cudaMemcpyAsync(M.active, M.hactive, sizeof(int) * B, cudaMemcpyHostToDevice, M.stream));
    void *e = nullptr;
    PMG_RET(vcycle(M, l0, B, c, minv, nullptr, &e));
    PMG_CUDA(M.h, k_update_u(M.L, g, H.pr, u1, s1, e, B, M.active));
    PMG_RET(norms(rn, nullptr));
    left = 0;
    for (int p = 0; p < B; ++p) {
      if (done[p]) continue;
      ++cyc[p];
      if (rn[p] >= o.mg_stall * r[p]) { done[p] = 1; continue; }
      r[p] = rn[p];
      if (!(r[p] > o.mg_tol * bn[p])) done[p] = 1;
      left += !done[p];
    }
  }
  int mx = 0;
  for (int p = 0; p < B; ++p) mx = cyc[p] > mx ? cyc[p] : mx;
  if (cycles) *cycles = mx;
  return PMG_OK;
}

MGCtx mgctx(pmg_ctx *h) {
  MGCtx M{h->L(), h->mgH ? h->mgH : &h->H, &h->opt, h->red, h->active, h->hred, h->hactive, h, h->stream, h->net};
  return M;
}

// ----------------------------------------------------------------- autotuner
//
// For every multigrid level (except the exact coarsest one) and both batch classes,
// time the candidate smoother variants -- one-point-per-thread kernels with 128, 256
// or 512 threads per block, and for 3D red-black Gauss-Seidel the fused z-marching
// sweep with z chunks of 8, 16 or 32 planes -- on the level's own buffers and keep the
// fastest.  Runs once at creation (it synchronises the stream).
// Candidates are timed the way the solver runs them: their sweeps captured into a CUDA
// graph (on a private stream, which waits for the work already on the solver's stream)
// and the graph replayed.  Timed eagerly, a variant of two launches per sweep (the
// one-point-per-thread kernels) paid the host's launch cost and lost on small grids to a
// fused sweep that is several times slower inside the graphs.
int autotune(MGCtx &M, int l0, int Bwide, double c) {
  Hier &H = *M.H;
  cudaEvent_t e0, e1;
  PMG_CUDA(M.h, cudaEventCreate(&e0));
  PMG_CUDA(M.h, cudaEventCreate(&e1));
  cudaStream_t ts = nullptr;
  PMG_CUDA(M.h, cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
  PMG_CUDA(M.h, cudaEventRecord(e0, M.stream));
  PMG_CUDA(M.h, cudaStreamWaitEvent(ts, e0, 0));
  MGCtx Mt = M;  // the same buffers, launched on ts, without profiling or launch counting
  Mt.L.stream = ts;
  Mt.L.counter = nullptr;
  Mt.L.prof = nullptr;
  Mt.stream = ts;
  constexpr int kSweeps = 4, kReplays = 5;  // sweeps per graph (the first from zero), timed replays
  int rc = PMG_OK;
  for (int l = l0; l < H.L - 1 && rc == PMG_OK; ++l)
    for (int cls = 0; cls < 2 && rc == PMG_OK; ++cls) {
      const int B = cls == 0 ? Bwide : 1;
      if (cls == 1 && Bwide == 1) { H.tune[l][1] = H.tune[l][0]; continue; }
      std::vector<Tune> cand;
      for (int th : {128, 256, 512}) cand.push_back(Tune{0, th, 256});
      const Grid &g = H.lev[l];
      if (M.o->smoother == PMG_SMOOTHER_RBGS && g.dim == 3 && g.n >= 15 && g.order != 4)
        for (int zc : {4, 8, 16, 32})  // short z chunks: more CTAs for single grids
          if (zc <= g.n) {
            cand.push_back(Tune{1, zc, 256});
            if (g.pitch >= 128) cand.push_back(Tune{1, zc, 512});
          }
      if (M.o->smoother == PMG_SMOOTHER_RBGS && rbgs_tma_supported(g, H.pr))
        for (int zc : {8, 16, 32, 64})
          if (zc <= g.n)
            for (int kind : {2, 3}) cand.push_back(Tune{kind, zc, rbgs_tma_threads(g, kind == 3)});
      float best = 1e30f;
      Tune pick = H.tune[l][cls];
      for (const Tune &t : cand) {
        void *cur = H.e[l];
        float ms = 0.f;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
          rc = fail(M.h, PMG_ERR_CUDA, "autotune capture failed");
          break;
        }
        for (int rep = 0; rep < kSweeps && rc == PMG_OK; ++rep) rc = smooth_with(Mt, t, l, B, c, cur, rep == 0);
        const cudaError_t ec = cudaStreamEndCapture(ts, &graph);
        if (rc != PMG_OK || ec != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          if (rc == PMG_OK) rc = fail(M.h, PMG_ERR_CUDA, "autotune capture failed");
          break;
        }
        bool ok = cudaGraphLaunch(exec, ts) == cudaSuccess && cudaEventRecord(e0, ts) == cudaSuccess;
        for (int r = 0; r < kReplays && ok; ++r) ok = cudaGraphLaunch(exec, ts) == cudaSuccess;
        ok = ok && cudaEventRecord(e1, ts) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
             cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (!ok) {
          rc = fail(M.h, PMG_ERR_CUDA, "autotune timing failed");
          break;
        }
        if (ms < best) { best = ms; pick = t; }
      }
      H.tune[l][cls] = pick;
    }
  if (cudaStreamSynchronize(ts) != cudaSuccess && rc == PMG_OK) rc = fail(M.h, PMG_ERR_CUDA, "autotune sync failed");
  cudaStreamDestroy(ts);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the timing sweeps left arbitrary values in the correction buffers; they are always
  // re-initialised before use, but clear them so the state is reproducible
  for (int l = l0; l < H.L && rc == PMG_OK; ++l) {
    const size_t bytes = (size_t)H.lev[l].slab * H.batch * H.tsize;
    if (cudaMemsetAsync(H.e[l], 0, bytes, M.stream) != cudaSuccess ||
        (H.e2[l] && cudaMemsetAsync(H.e2[l], 0, bytes, M.stream) != cudaSuccess))
      rc = fail(M.h, PMG_ERR_CUDA, "autotune clear failed");
  }
  return rc;
}

// ----------------------------------------------------------------- SDC / PFASST schedule

// With fixed V-cycle counts the fine level keeps no F = A U array: the end-of-iteration
// pass (fine_residual) evaluates F from U, forms the collocation residual and the
// right-hand sides q of the next fine sweep; the FAS restriction evaluates the fine F
// at the coarse points only.  On GB300, whose FP64 rate is a small fraction of its FP32
// rate, this removes most FP64 stencil work.  Full solves keep F (their sub-step
// residuals need b = u_m + q_m).
bool ffree(const pmg_ctx *h) { return h->opt.vcycles > 0; }

// collocation residual of the fine level into red[2P..3P) (+ next right-hand sides
// when F-free), copied to hred asynchronously; `chained` right after a send-forward
int fine_residual(pmg_ctx *h, bool chained = false) {
  const long long sfs = (long long)h->sf * h->gf.slab;
  PMG_CUDA(h, cudaMemsetAsync(h->red + 2 * h->P, 0, sizeof(unsigned long long) * h->P, h->stream));
  if (ffree(h))
    PMG_CUDA(h, k_fine_rhs_residual(h->L(), h->gf, h->resf, h->nu, h->Uf, sfs, h->qf, (long long)(h->sf - 1) * h->gf.slab,
                                    h->P, h->red + 2 * h->P, chained));
  else
    PMG_CUDA(h, k_colloc_residual(h->L(), h->gf, h->resf, h->Uf, h->Ff, sfs, h->P, h->red + 2 * h->P));
  if (!h->in_loop)  // the device-side loop keeps the residual on the device (loop_check_kernel)
    PMG_CUDA(h, cudaMemcpyAsync(h->hred + 2 * h->P, h->red + 2 * h->P, sizeof(unsigned long long) * h->P,
                                cudaMemcpyDeviceToHost, h->stream));
  return PMG_OK;
}

// The state of one level of the hierarchy (0 fine, 1 coarse, 2 coarsest of three);
// level l lives on multigrid level l of the hierarchy H (grid n_l = (n_{l-1}-1)/2)
struct LevelRef {
  const Grid *g;
  int s;                        // nodes
  double *U, *F, *q, *tau;      // tau: FAS correction (null on the fine level)
  const SFCoef *cf;
  const double *csub;           // c_m = dt_m nu per sub-step
  int slot0;                    // coarsest-grid inverse of its first sub-step
};

LevelRef level_ref(pmg_ctx *h, int level) {
  if (level == 0) return LevelRef{&h->gf, h->sf, h->Uf, h->Ff, h->qf, nullptr, &h->sff, h->cf_sub, 0};
  if (level == 1) return LevelRef{&h->gc, h->sc, h->Uc, h->Fc, h->qc, h->tau, &h->sfc, h->cc_sub, h->sf - 1};
  return LevelRef{&h->g2, h->s2, h->U2, h->F2, h->q2, h->tau2, &h->sf2c, h->c2_sub, (h->sf - 1) + (h->sc - 1)};
}

// One SDC sweep (Eq. sdc-be) on slices [p0, p0+B) of `level`.  Coarser levels keep
// F = A U and add their FAS correction; F-free fine sweeps take q from the last
// fine_residual.
int sweep(pmg_ctx *h, int level, int p0, int B) {
  MGCtx M = mgctx(h);
  if (level > 0) M.o = &h->opt_c;  // the coarse levels' sub-step solver (coarse_vcycles)
  const LevelRef v = level_ref(h, level);
  const Grid &g = *v.g;
  const long long stride = (long long)v.s * g.slab, sq = (long long)(v.s - 1) * g.slab;
  double *U = v.U + p0 * stride;
  double *F = v.F ? v.F + p0 * stride : nullptr;  // null: F-free fine level
  double *q = v.q + p0 * sq;
  const double *tau = v.tau ? v.tau + p0 * stride : nullptr;
  const bool keepF = level > 0 || !ffree(h);
  Launch Ln = h->L();
  if (keepF) PMG_CUDA(h, k_sf_rhs(Ln, g, *v.cf, F, U, stride, tau, stride, q, sq, B));
  for (int m = 0; m < v.s - 1; ++m) {
    PMG_RET(solve_substep(M, level, B, v.csub[m], h->minv_slot(v.slot0 + m), U + m * g.slab, stride, q + m * g.slab,
                          sq, U + (m + 1) * g.slab, stride, nullptr, v.cf->sub_next != 0));
    if (keepF) PMG_CUDA(h, k_apply_A(Ln, g, h->nu, U + (m + 1) * g.slab, stride, F + (m + 1) * g.slab, stride, B));
  }
  return PMG_OK;
}

int fas_restrict_all(pmg_ctx *h) {
  const long long sfs = (long long)h->sf * h->gf.slab, scs = (long long)h->sc * h->gc.slab;
  if (ffree(h))
    PMG_CUDA(h, k_fas_restrict_u(h->L(), h->gf, h->gc, h->fas, h->Uf, sfs, h->Uc, h->Fc, h->tau, h->Uc0, scs, h->P));
  else
    PMG_CUDA(h, k_fas_restrict(h->L(), h->gf, h->gc, h->fas, h->Uf, h->Ff, sfs, h->Uc, h->Fc, h->tau, h->Uc0, scs,
                               h->P));
  return PMG_OK;
}

// FAS restriction level 1 -> 2 of every slice: level 1 keeps F = A U, and its own
// FAS correction enters the integral it passes down
int fas_restrict_12(pmg_ctx *h) {
  const long long s1 = (long long)h->sc * h->gc.slab, s2 = (long long)h->s2 * h->g2.slab;
  PMG_CUDA(h, k_fas_restrict(h->L(), h->gc, h->g2, h->fas2, h->Uc, h->Fc, s1, h->U2, h->F2, h->tau2, h->U20, s2, h->P,
                             h->tau));
  return PMG_OK;
}

// U_l[p][0] <- U_l[p-1][s_l - 1] and F_l[p][0] = A_l U_l[p][0] for p in [p0, p0+B),
// p0 >= 1, on a coarse level l.  A coarse level keeps F_l = A_l U_l at every node, so
// F_l[p-1][s_l - 1] already is A_l applied to the received value: it is copied instead
// of evaluated again (bitwise the same numbers, no FP64 stencil).
int receive(pmg_ctx *h, int level, int p0, int B) {
  const LevelRef v = level_ref(h, level);
  const long long st = (long long)v.s * v.g->slab, last = (long long)(v.s - 1) * v.g->slab;
  PMG_CUDA(h, k_copy(h->L(), *v.g, v.U + (p0 - 1) * st + last, st, v.U + p0 * st, st, B));
  PMG_CUDA(h, k_copy(h->L(), *v.g, v.F + (p0 - 1) * st + last, st, v.F + p0 * st, st, B));
  return PMG_OK;
}

// the serial chain on the coarsest level: slice p receives the end value of slice p-1
// (the blocking coarse communication of Sec. 2.4), then sweeps
int coarse_chain(pmg_ctx *h) {
  const int lc = h->nlevels - 1;
  for (int p = 0; p < h->P; ++p) {
    if (p > 0) PMG_RET(receive(h, lc, p, 1));
    PMG_RET(sweep(h, lc, p, 1));
  }
  return PMG_OK;
}

// correction of level 2 interpolated onto every node of level 1.  Node 0 is included:
// for slices p >= 1 the received coarsest initial value moves it, and through the
// level-1 Lagrange weights it reaches fine nodes that no send-forward overwrites.
// F_1 is left stale: nothing reads it before the next restriction from level 0
// rewrites it.
int interp_21(pmg_ctx *h) {
  const long long s1 = (long long)h->sc * h->gc.slab, s2 = (long long)h->s2 * h->g2.slab;
  PMG_CUDA(h, k_interp_time(h->L(), h->g2, h->interp2, h->H.pr, h->U2, h->U20, s2, h->dU2, h->P, 0));
  PMG_CUDA(h, k_interp_space_add(h->L(), h->gc, h->g2, h->opt.interp_order, h->sc, h->H.pr, h->dU2, h->Uc, s1, h->P,
                                 0));
  return PMG_OK;
}

// m0 = 1 inside an iteration: the send-forward that follows overwrites node 0 of slices
// p >= 1, and for slice 0 the coarse correction at node 0 is exactly zero (its coarse
// node 0 is the restricted initial value, which no sweep changes)
int interp_all(pmg_ctx *h, int m0 = 0) {
  const long long sfs = (long long)h->sf * h->gf.slab, scs = (long long)h->sc * h->gc.slab;
  PMG_CUDA(h, k_interp_time(h->L(), h->gc, h->interp, h->H.pr, h->Uc, h->Uc0, scs, h->dU, h->P, m0));
  PMG_CUDA(h, k_interp_space_add(h->L(), h->gf, h->gc, h->opt.interp_order, h->sf, h->H.pr, h->dU, h->Uf, sfs, h->P,
                                 m0));
  if (!ffree(h)) PMG_CUDA(h, k_apply_A(h->L(), h->gf, h->nu, h->Uf, h->gf.slab, h->Ff, h->gf.slab, h->P * h->sf));
  return PMG_OK;
}

// elapsed times of the event nodes of the last replay of a graph
int harvest(pmg_ctx *h, pmg_ctx::Captured &G) {
  for (const ProfRec &r : G.recs) {
    float ms = 0.f;
    PMG_CUDA(h, cudaEventElapsedTime(&ms, r.a, r.b));
    h->prof.done.push_back(ProfDone{r.kid, r.n, r.prec, r.pts, ms});
  }
  return PMG_OK;
}

void drop_graph(pmg_ctx::Captured &G) {
  if (G.exec) cudaGraphExecDestroy(G.exec);
  G.exec = nullptr;
  G.recs.clear();
}

// run body on the caller's stream through a CUDA graph captured on a private stream
// (captured again when the profiling settings changed since the last capture)
int run_graph(pmg_ctx *h, pmg_ctx::Captured &G, int (*body)(pmg_ctx *)) {
  if (G.exec && (G.with_prof != h->prof.on || G.prof_min != h->prof.min_points)) drop_graph(G);
  if (!G.exec) {
    if (!h->cap_stream) PMG_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = h->stream;
    const long long before = h->launches;
    h->stream = h->cap_stream;
    h->prof.capture = &G.recs;
    G.recs.clear();
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    int rc = e == cudaSuccess ? body(h) : PMG_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(h->cap_stream, &graph) : e;
    h->stream = user;
    h->prof.capture = nullptr;
    G.kernels = h->launches - before;
    h->launches = before;
    if (rc != PMG_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (e2 != cudaSuccess) return fail(h, PMG_ERR_CUDA, std::string("stream capture: ") + cudaGetErrorString(e2));
    // per-node priorities: the coarse-chain kernels keep the high priority of their stream
    e = cudaGraphInstantiate(&G.exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { G.exec = nullptr; return fail(h, PMG_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e)); }
    G.with_prof = h->prof.on;
    G.prof_min = h->prof.min_points;
  }
  PMG_CUDA(h, cudaGraphLaunch(G.exec, h->stream));
  h->launches += G.kernels;
  return PMG_OK;
}

bool use_graphs(const pmg_ctx *h) { return h->opt.use_graphs && h->opt.vcycles > 0 && h->opt_c.vcycles > 0; }

// predictor (Sec. 2.4): restrict down to the coarsest level, P stages there (stage s
// sweeps slices s..P-1 after they received the end values of s-1..P-2), interpolate up
int predict_body(pmg_ctx *h) {
  if (h->nlevels >= 2) {
    const int lc = h->nlevels - 1;
    PMG_RET(fas_restrict_all(h));
    if (h->nlevels == 3) PMG_RET(fas_restrict_12(h));
    for (int s = 0; s < h->P; ++s) {
      if (s > 0) PMG_RET(receive(h, lc, s, h->P - s));
      PMG_RET(sweep(h, lc, s, h->P - s));
    }
    if (h->nlevels == 3) PMG_RET(interp_21(h));
    PMG_RET(interp_all(h));
  }
  return ffree(h) ? fine_residual(h) : PMG_OK;  // right-hand sides of the first fine sweep
}

// The predictor right after a spread.  Every slice then starts from the same values,
// and FAS restricts identical fine states to identical coarse states and FAS terms, so
// before stage s all slices p >= s hold one and the same state A_s: stage s computes
// one sweep of A_s (with node 0 replaced by its own end value) P - s times over.  Slice
// p keeps A_{p+1}.  The same numbers come from a serial chain: slice s takes the state
// of slice s-1 (its final A_s), receives slice s-1's end value at node 0 and sweeps
// once -- P single-slice sweeps instead of P (P + 1) / 2 slice-sweeps in P stages.
int predict_body_spread(pmg_ctx *h) {
  if (h->nlevels >= 2) {
    const int lc = h->nlevels - 1;
    PMG_RET(fas_restrict_all(h));
    if (h->nlevels == 3) PMG_RET(fas_restrict_12(h));
    const LevelRef v = level_ref(h, lc);
    const long long st = (long long)v.s * v.g->slab;
    for (int s = 0; s < h->P; ++s) {
      if (s > 0) {  // nodes 1..M of slice s-1, then node 0 received from its end
        PMG_CUDA(h, k_copy(h->L(), *v.g, v.U + (s - 1) * st + v.g->slab, v.g->slab, v.U + s * st + v.g->slab,
                           v.g->slab, v.s - 1));
        PMG_CUDA(h, k_copy(h->L(), *v.g, v.F + (s - 1) * st + v.g->slab, v.g->slab, v.F + s * st + v.g->slab,
                           v.g->slab, v.s - 1));
        PMG_RET(receive(h, lc, s, 1));
      }
      PMG_RET(sweep(h, lc, s, 1));
    }
    if (h->nlevels == 3) PMG_RET(interp_21(h));
    PMG_RET(interp_all(h));
  }
  return ffree(h) ? fine_residual(h) : PMG_OK;
}

int predict(pmg_ctx *h) {
  const bool fast = h->spread_state;
  pmg_ctx::Captured &G = fast ? h->g_pred_spread : h->g_pred;
  int (*body)(pmg_ctx *) = fast ? predict_body_spread : predict_body;
  if (use_graphs(h)) {
    PMG_RET(run_graph(h, G, body));
    if (!G.recs.empty()) {
      PMG_CUDA(h, cudaStreamSynchronize(h->stream));
      PMG_RET(harvest(h, G));
    }
  } else {
    PMG_RET(body(h));
  }
  h->spread_state = false;
  h->predicted = true;
  h->q_valid = ffree(h);
  return PMG_OK;
}

// ---- pieces of one PFASST iteration on the slices [p0, p0+B)

int fas_part(pmg_ctx *h, int p0, int B) {
  const long long sfs = (long long)h->sf * h->gf.slab, scs = (long long)h->sc * h->gc.slab;
  PMG_CUDA(h, k_fas_restrict_u(h->L(), h->gf, h->gc, h->fas, h->Uf + p0 * sfs, sfs, h->Uc + p0 * scs,
                               h->Fc + p0 * scs, h->tau + p0 * scs, h->Uc0 + p0 * scs, scs, B));
  return PMG_OK;
}

int interp_part(pmg_ctx *h, int p0, int B) {
  const long long sfs = (long long)h->sf * h->gf.slab, scs = (long long)h->sc * h->gc.slab;
  void *dU = (char *)h->dU + (size_t)p0 * h->sf * h->gc.slab * h->H.tsize;
  PMG_CUDA(h, k_interp_time(h->L(), h->gc, h->interp, h->H.pr, h->Uc + p0 * scs, h->Uc0 + p0 * scs, scs, dU, B, 1));
  PMG_CUDA(h, k_interp_space_add(h->L(), h->gf, h->gc, h->opt.interp_order, h->sf, h->H.pr, dU, h->Uf + p0 * sfs,
                                 sfs, B, 1));
  return PMG_OK;
}

// U_f[p][0] <- U_f[p-1][M_f] for p in [max(p0,1), p0+B)
int send_forward_part(pmg_ctx *h, int p0, int B) {
  const long long sfs = (long long)h->sf * h->gf.slab;
  const int first = p0 > 1 ? p0 : 1, cnt = p0 + B - first;
  if (cnt > 0)
    PMG_CUDA(h, k_copy(h->L(), h->gf, h->Uf + (first - 1) * sfs + (h->sf - 1) * h->gf.slab, sfs,
                       h->Uf + first * sfs, sfs, cnt));
  return PMG_OK;
}

// F-free fine level: collocation residual and next right-hand sides of [p0, p0+B)
int fine_residual_part(pmg_ctx *h, int p0, int B) {
  const long long sfs = (long long)h->sf * h->gf.slab, sq = (long long)(h->sf - 1) * h->gf.slab;
  PMG_CUDA(h, k_fine_rhs_residual(h->L(), h->gf, h->resf, h->nu, h->Uf + p0 * sfs, sfs, h->qf + p0 * sq, sq, B,
                                  h->red + 2 * h->P + p0, true));
  return PMG_OK;
}

// One PFASST iteration with the slices in `groups` groups (Sec. 2.4 schedule, same
// operations on the same data as iteration_serial, so the results are identical):
//   main stream:  fine sweep + FAS restriction of group 0, 1, ...
//   chain stream: as soon as group g is restricted, the coarse sweeps of its slices in
//                 order (slice p receives the coarse end value of p-1) -- the serial
//                 part, overlapped with the fine sweeps of the later groups
//   post stream:  as soon as the chain has passed group g, its interpolation,
//                 send-forward and collocation residual / next right-hand sides
int iteration_pipe(pmg_ctx *h) {
  const int P = h->P, G = h->groups, per = (P + G - 1) / G;
  cudaStream_t main = h->stream;
  PMG_CUDA(h, cudaMemsetAsync(h->red + 2 * P, 0, sizeof(unsigned long long) * P, main));
  PMG_CUDA(h, cudaEventRecord(h->ev_fork, main));
  PMG_CUDA(h, cudaStreamWaitEvent(h->s_chain, h->ev_fork, 0));
  PMG_CUDA(h, cudaStreamWaitEvent(h->s_post, h->ev_fork, 0));
  auto group = [&](int g, int &p0, int &B) {
    p0 = g * per;
    B = P - p0 < per ? P - p0 : per;
    return B > 0;
  };
  int rc = PMG_OK;
  int p0 = 0, B = 0;
  for (int g = 0; g < G && rc == PMG_OK && group(g, p0, B); ++g) {
    rc = sweep(h, 0, p0, B);
    if (rc == PMG_OK) rc = fas_part(h, p0, B);
    if (rc == PMG_OK && cudaEventRecord(h->ev_fas[g], h->stream) != cudaSuccess)
      rc = fail(h, PMG_ERR_CUDA, "event record failed");
  }
  h->stream = h->s_chain;
  h->mgH = &h->Hc;
  for (int g = 0; g < G && rc == PMG_OK && group(g, p0, B); ++g) {
    if (cudaStreamWaitEvent(h->stream, h->ev_fas[g], 0) != cudaSuccess) rc = fail(h, PMG_ERR_CUDA, "wait failed");
    for (int p = p0; p < p0 + B && rc == PMG_OK; ++p) {
      if (p > 0) rc = receive(h, 1, p, 1);
      if (rc == PMG_OK) rc = sweep(h, 1, p, 1);
    }
    if (rc == PMG_OK && cudaEventRecord(h->ev_chain[g], h->stream) != cudaSuccess)
      rc = fail(h, PMG_ERR_CUDA, "event record failed");
  }
  h->mgH = nullptr;
  if (rc == PMG_OK && cudaEventRecord(h->ev_chain_end, h->stream) != cudaSuccess)
    rc = fail(h, PMG_ERR_CUDA, "event record failed");
  h->stream = h->s_post;
  for (int g = 0; g < G && rc == PMG_OK && group(g, p0, B); ++g) {
    if (cudaStreamWaitEvent(h->stream, h->ev_chain[g], 0) != cudaSuccess) rc = fail(h, PMG_ERR_CUDA, "wait failed");
    if (rc == PMG_OK) rc = interp_part(h, p0, B);
    if (rc == PMG_OK) rc = send_forward_part(h, p0, B);
    if (rc == PMG_OK) rc = fine_residual_part(h, p0, B);
  }
  if (rc == PMG_OK && cudaEventRecord(h->ev_post_end, h->stream) != cudaSuccess)
    rc = fail(h, PMG_ERR_CUDA, "event record failed");
  h->stream = main;
  // join both side streams (also required to end a stream capture)
  PMG_CUDA(h, cudaStreamWaitEvent(main, h->ev_chain_end, 0));
  PMG_CUDA(h, cudaStreamWaitEvent(main, h->ev_post_end, 0));
  if (rc != PMG_OK) return rc;
  PMG_CUDA(h, cudaMemcpyAsync(h->hred + 2 * P, h->red + 2 * P, sizeof(unsigned long long) * P,
                              cudaMemcpyDeviceToHost, main));
  return PMG_OK;
}

// one PFASST iteration (Sec. 2.4), residual copied to hred[2P..3P) asynchronously.
// With three levels: fine sweep, restriction, level-1 sweep on every slice at once,
// restriction, serial chain on level 2, corrections interpolated level by level up
int iteration(pmg_ctx *h) {
  // (a deployed network shares one scratch between all V-cycles: no overlap then)
  if (h->groups > 1 && !h->net) return iteration_pipe(h);
  const long long sfs = (long long)h->sf * h->gf.slab;
  PMG_RET(sweep(h, 0, 0, h->P));
  if (h->nlevels >= 2) {
    PMG_RET(fas_restrict_all(h));
    if (h->nlevels == 3) {
      PMG_RET(sweep(h, 1, 0, h->P));
      PMG_RET(fas_restrict_12(h));
    }
    PMG_RET(coarse_chain(h));
    if (h->nlevels == 3) PMG_RET(interp_21(h));
    PMG_RET(interp_all(h, 1));
  }
  if (h->P > 1) {  // send forward: U_f[p][0] <- U_f[p-1][M_f]
    PMG_CUDA(h, k_copy(h->L(), h->gf, h->Uf + (h->sf - 1) * h->gf.slab, sfs, h->Uf + sfs, sfs, h->P - 1));
    // with a stored F, F_f[p][M_f] = A U_f[p][M_f] already (interpolation re-evaluates it)
    if (!ffree(h))
      PMG_CUDA(h, k_copy(h->L(), h->gf, h->Ff + (h->sf - 1) * h->gf.slab, sfs, h->Ff + sfs, sfs, h->P - 1));
  }
  return fine_residual(h, true);
}

// End of one iteration of the device-side loop (one warp): the collocation residual of
// the iteration (max over slices of the per-slice maxima, as bit patterns of
// non-negative doubles, so Inf and NaN compare largest), the iteration count, and
// whether the loop goes on: fewer than max_iter iterations, residual above tol and
// finite.
__global__ void loop_check_kernel(const unsigned long long *__restrict__ res, int P, LoopCtl *ctl,
                                  cudaGraphConditionalHandle cond) {
  unsigned long long mx = 0ULL;
  for (int p = threadIdx.x; p < P; p += 32) mx = res[p] > mx ? res[p] : mx;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = w > mx ? w : mx;
  }
  if (threadIdx.x == 0) {
    const int k = ctl->k + 1;
    ctl->k = k;
    ctl->res_bits = mx;
    const bool finite = mx < 0x7ff0000000000000ULL;
    const bool go = k < ctl->max_iter && finite && !(__longlong_as_double((long long)mx) <= ctl->tol);
    cudaGraphSetConditional(cond, go ? 1u : 0u);
  }
}

// The PFASST iteration loop as one CUDA graph: a conditional while-node whose body is
// one iteration (captured once) followed by loop_check_kernel, which decides on the
// device whether the body runs again.  One graph launch runs the whole loop with no
// host round trip between iterations.  Conditional bodies hold no event nodes, so this
// serves the single-stream schedule without the launch profiler.
bool device_loop_ok(const pmg_ctx *h) { return use_graphs(h) && h->groups == 1 && !h->prof.on; }

int build_loop_graph(pmg_ctx *h) {
  if (!h->cap_stream) PMG_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  PMG_CUDA(h, cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};  // remaining members zero
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return fail(h, PMG_ERR_CUDA, std::string("conditional graph node: ") + cudaGetErrorString(e));
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t user = h->stream;
  const long long before = h->launches;
  h->stream = h->cap_stream;
  h->in_loop = true;
  e = cudaStreamBeginCaptureToGraph(h->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  int rc = e == cudaSuccess ? iteration(h) : PMG_ERR_CUDA;
  if (rc == PMG_OK) {
    loop_check_kernel<<<1, 32, 0, h->cap_stream>>>(h->red + 2 * h->P, h->P, h->ctl, cond);
    if (cudaGetLastError() != cudaSuccess) rc = fail(h, PMG_ERR_CUDA, "loop check launch failed");
    ++h->launches;
  }
  cudaGraph_t body_out = nullptr;
  cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(h->cap_stream, &body_out) : e;
  h->stream = user;
  h->in_loop = false;
  h->g_loop.kernels = h->launches - before;
  h->launches = before;
  if (rc == PMG_OK && e2 != cudaSuccess)
    rc = fail(h, PMG_ERR_CUDA, std::string("loop body capture: ") + cudaGetErrorString(e2));
  if (rc == PMG_OK) {
    e = cudaGraphInstantiate(&h->g_loop.exec, graph, 0);
    if (e != cudaSuccess) {
      h->g_loop.exec = nullptr;
      rc = fail(h, PMG_ERR_CUDA, std::string("cudaGraphInstantiate (loop): ") + cudaGetErrorString(e));
    }
  }
  cudaGraphDestroy(graph);
  return rc;
}

// run up to max_iter iterations (>= 1) on the device; *k and *res receive the
// iterations done and the last residual
int run_device_loop(pmg_ctx *h, int max_iter, double tol, int *k, double *res) {
  if (!h->g_loop.exec) PMG_RET(build_loop_graph(h));
  h->hctl->max_iter = max_iter;
  h->hctl->k = 0;
  h->hctl->tol = tol;
  h->hctl->res_bits = 0ULL;
  PMG_CUDA(h, cudaMemcpyAsync(h->ctl, h->hctl, sizeof(LoopCtl), cudaMemcpyHostToDevice, h->stream));
  PMG_CUDA(h, cudaGraphLaunch(h->g_loop.exec, h->stream));
  PMG_CUDA(h, cudaMemcpyAsync(h->hctl, h->ctl, sizeof(LoopCtl), cudaMemcpyDeviceToHost, h->stream));
  PMG_CUDA(h, cudaStreamSynchronize(h->stream));
  *k = h->hctl->k;
  std::memcpy(res, &h->hctl->res_bits, 8);
  h->launches += h->g_loop.kernels * (long long)*k;
  return PMG_OK;
}

double bits_to_double(unsigned long long v) {
  double d;
  std::memcpy(&d, &v, 8);
  return d;
}

int spread(pmg_ctx *h) {
  // copy u0 to every node of every slice; with a stored F, also F = A u0 everywhere
  if (!ffree(h)) {
    PMG_CUDA(h, k_apply_A(h->L(), h->gf, h->nu, h->u0, 0, h->dense, 0, 1));
    PMG_CUDA(h, k_copy(h->L(), h->gf, h->dense, 0, h->Ff, h->gf.slab, h->P * h->sf));
  }
  PMG_CUDA(h, k_copy(h->L(), h->gf, h->u0, 0, h->Uf, h->gf.slab, h->P * h->sf));
  h->predicted = false;
  h->q_valid = false;
  h->spread_state = true;
  return PMG_OK;
}

void fill_coefficients(pmg_ctx *h) {
  long double Qf[kMaxNodes][kMaxNodes], Qc[kMaxNodes][kMaxNodes];
  node_positions(h->sf, h->famf, h->tauf);
  integration_matrix(h->sf, h->tauf, Qf, h->famf);
  auto fill_sf = [&](SFCoef &cf, int s, const long double *t, long double Q[kMaxNodes][kMaxNodes], double *csub,
                     int vcycles) {
    std::memset(&cf, 0, sizeof cf);
    cf.s = s;
    cf.sub_next = vcycles > 0;  // fixed V-cycle counts start from the pointwise residual
    for (int m = 0; m < s - 1; ++m) {
      const long double dtm = (long double)h->dt * (t[m + 1] - t[m]);
      csub[m] = (double)(dtm * h->nu);
      for (int j = 0; j < s; ++j) {
        long double w = (long double)h->dt * (Q[m + 1][j] - Q[m][j]);
        if (j == m + 1 && !cf.sub_next) w -= dtm;
        cf.W[m][j] = (double)w;
      }
    }
  };
  fill_sf(h->sff, h->sf, h->tauf, Qf, h->cf_sub, h->opt.vcycles);
  std::memset(&h->resf, 0, sizeof h->resf);
  h->resf.s = h->sf;
  for (int m = 0; m < h->sf; ++m)
    for (int i = 0; i < h->sf; ++i) {
      h->resf.dtQ[m][i] = (double)((long double)h->dt * Qf[m][i]);
      if (m + 1 < h->sf) h->resf.dS[m][i] = (double)((long double)h->dt * (Qf[m + 1][i] - Qf[m][i]));
    }
  // restriction from a level with s nodes t (integration matrix Q) to one with sc nodes
  // tc (Qc): map[j] = the finer node at the time of coarse node j (-1: none)
  auto fill_fas = [&](FASCoef &cf, int s, const long double *t, long double Q[kMaxNodes][kMaxNodes], int sc,
                      const long double *tc, long double Qcc[kMaxNodes][kMaxNodes]) {
    std::memset(&cf, 0, sizeof cf);
    cf.sf = s;
    cf.sc = sc;
    cf.nu = h->nu;
    for (int j = 0; j < sc; ++j) {
      cf.map[j] = -1;
      for (int m = 0; m < s; ++m)
        if (fabsl(t[m] - tc[j]) < 1e-13L) cf.map[j] = m;
      if (cf.map[j] < 0) continue;  // rejected at creation
      for (int i = 0; i < s; ++i) cf.dtQf[j][i] = (double)((long double)h->dt * Q[cf.map[j]][i]);
      for (int i = 0; i < sc; ++i) cf.dtQc[j][i] = (double)((long double)h->dt * Qcc[j][i]);
    }
  };
  auto fill_interp = [&](InterpCoef &ic, int s, const long double *t, int sc, const long double *tc) {
    std::memset(&ic, 0, sizeof ic);
    ic.sf = s;
    ic.sc = sc;
    ic.order = h->opt.interp_order;
    for (int m = 0; m < s; ++m) {
      lagrange_row(sc, tc, t[m], ic.T[m]);
      for (int j = 0; j < sc; ++j) ic.T32[m][j] = (float)ic.T[m][j];
    }
  };
  if (h->nlevels >= 2) {
    node_positions(h->sc, h->famc, h->tauc);
    integration_matrix(h->sc, h->tauc, Qc, h->famc);
    fill_sf(h->sfc, h->sc, h->tauc, Qc, h->cc_sub, h->opt_c.vcycles);
    fill_fas(h->fas, h->sf, h->tauf, Qf, h->sc, h->tauc, Qc);
    fill_interp(h->interp, h->sf, h->tauf, h->sc, h->tauc);
  }
  if (h->nlevels == 3) {
    long double Q2[kMaxNodes][kMaxNodes];
    node_positions(h->s2, h->fam2, h->tau2n);
    integration_matrix(h->s2, h->tau2n, Q2, h->fam2);
    fill_sf(h->sf2c, h->s2, h->tau2n, Q2, h->c2_sub, h->opt_c.vcycles);
    fill_fas(h->fas2, h->sc, h->tauc, Qc, h->s2, h->tau2n, Q2);
    fill_interp(h->interp2, h->sc, h->tauc, h->s2, h->tau2n);
  }
}

int upload_minv(pmg_ctx *h) {
  const int slots = minv_slots(h);
  std::vector<double> M;
  std::vector<char> buf((size_t)slots * h->n3 * h->n3 * h->H.tsize);
  for (int s = 0; s < slots; ++s) {
    const int s1 = h->sf - 1, s12 = s1 + (h->sc > 0 ? h->sc - 1 : 0);
    const double c = s < s1 ? h->cf_sub[s] : (s < s12 ? h->cc_sub[s - s1] : h->c2_sub[s - s12]);
    coarsest_inverse(h->dim, c, M);
    for (size_t q = 0; q < M.size(); ++q) {
      char *dst = buf.data() + ((size_t)s * h->n3 * h->n3 + q) * h->H.tsize;
      if (h->H.tsize == 8) std::memcpy(dst, &M[q], 8);
      else { float fv = (float)M[q]; std::memcpy(dst, &fv, 4); }
    }
  }
  PMG_CUDA(h, cudaMemcpyAsync(h->minv, buf.data(), buf.size(), cudaMemcpyHostToDevice, h->stream));
  PMG_CUDA(h, cudaStreamSynchronize(h->stream));
  return PMG_OK;
}

pmg_ctx *make_ctx(const pmg_grid *grid, const pmg_nodes_desc *fn, const pmg_levels *lv, double nu, double dt,
                  int slices, const pmg_options *opt) {
  pmg_ctx *h = new (std::nothrow) pmg_ctx();
  if (!h) return nullptr;
  if (opt) h->opt = *opt; else pfasst_mg_default_options(&h->opt);
  h->opt_c = h->opt;
  if (h->opt.coarse_vcycles >= 0) h->opt_c.vcycles = h->opt.coarse_vcycles;
  h->dim = grid->dim;
  h->nf = grid->n;
  h->nc = (grid->n - 1) / 2;
  h->sf = fn->count;
  h->famf = fn->family;
  h->famc = lv->nlevels >= 2 ? lv->coarse_nodes.family : 0;
  h->fam2 = lv->nlevels == 3 ? lv->coarsest_nodes.family : 0;
  h->nlevels = lv->nlevels;
  h->sc = lv->nlevels >= 2 ? lv->coarse_nodes.count : 0;
  h->s2 = lv->nlevels == 3 ? lv->coarsest_nodes.count : 0;
  h->P = slices;
  h->nu = nu;
  h->dt = dt;
  h->order = grid_order(grid);
  h->gf = make_grid(h->dim, h->nf, h->order);
  if (h->nlevels >= 2) h->gc = make_grid(h->dim, h->nc);
  if (h->nlevels == 3) h->g2 = make_grid(h->dim, (h->nc - 1) / 2);
  h->n3 = h->dim == 1 ? 3 : (h->dim == 2 ? 9 : 27);
  // slice groups: only two-level PFASST with fixed V-cycle counts pipelines (with three
  // levels the chain runs on level 2 after a batched level-1 sweep)
  int G = h->opt.slice_groups;
  // automatic: no overlap.  On the 3D workload 2 groups gain 1.5 % (every fine kernel
  // already fills the GPU), and overlapping kernels blur per-kernel timings.
  if (G == 0) G = 1;
  if (G > slices) G = slices;
  h->groups = (h->nlevels == 2 && h->opt.vcycles > 0 && h->opt_c.vcycles > 0 && G > 1) ? G : 1;
  return h;
}

}  // namespace

// ----------------------------------------------------------------- C ABI

extern "C" {

void pfasst_mg_default_options(pmg_options *o) {
  if (!o) return;
  o->smoother = PMG_SMOOTHER_JACOBI;
  o->omega = 2.0 / 3.0;
  o->nu1 = 2;
  o->nu2 = 1;
  o->vcycles = 2;
  o->mg_tol = 1e-12;
  o->mg_stall = 0.75;
  o->mg_maxcycles = 50;
  o->precision = PMG_PREC_FP64;
  o->interp_order = 4;
  o->use_graphs = 1;
  o->autotune = 1;
  o->slice_groups = 0;
  o->vcycle_tail = -1;
  o->coarse_vcycles = -1;
  o->single_grid_vcycle = 0;
}

int pfasst_mg_workspace_bytes(const pmg_grid *grid, const pmg_nodes_desc *fn, const pmg_levels *lv, int slices,
                              const pmg_options *opt, size_t *bytes) {
  std::string why;
  int rc = validate(grid, fn, lv, slices, opt, why);
  if (rc != PMG_OK) return fail(nullptr, rc, why);
  if (!bytes) return fail(nullptr, PMG_ERR_INVALID_ARG, "bytes is null");
  pmg_ctx *h = make_ctx(grid, fn, lv, 1.0, 1.0, slices, opt);
  if (!h) return fail(nullptr, PMG_ERR_OOM, "host allocation failed");
  Plan pl;
  plan_ctx(pl, h);
  *bytes = pl.total;
  delete h;
  return PMG_OK;
}

int pfasst_mg_create(const pmg_grid *grid, const pmg_nodes_desc *fn, const pmg_levels *lv, double nu, double dt,
                     int slices, const pmg_options *opt, void *stream, void *workspace, size_t workspace_bytes,
                     pmg_handle *out) {
  if (!out) return fail(nullptr, PMG_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  std::string why;
  int rc = validate(grid, fn, lv, slices, opt, why);
  if (rc != PMG_OK) return fail(nullptr, rc, why);
  if (!(nu > 0) || !(dt > 0) || !std::isfinite(nu) || !std::isfinite(dt))
    return fail(nullptr, PMG_ERR_INVALID_ARG, "nu and dt must be positive and finite");
  pmg_ctx *h = make_ctx(grid, fn, lv, nu, dt, slices, opt);
  if (!h) return fail(nullptr, PMG_ERR_OOM, "host allocation failed");
  h->stream = (cudaStream_t)stream;
  fill_coefficients(h);
  bool nested = true;
  for (int j = 0; j < h->sc && h->nlevels >= 2; ++j) nested = nested && h->fas.map[j] >= 0;
  if (!nested) {
    delete h;
    return fail(nullptr, PMG_ERR_INVALID_ARG, "coarse nodes are not a subset of the fine nodes");
  }
  for (int j = 0; j < h->s2 && h->nlevels == 3; ++j) nested = nested && h->fas2.map[j] >= 0;
  if (!nested) {
    delete h;
    return fail(nullptr, PMG_ERR_INVALID_ARG, "coarsest nodes are not a subset of the coarse nodes");
  }
  Plan pl;
  plan_ctx(pl, h);
  if (workspace) {
    if (workspace_bytes < pl.total || ((uintptr_t)workspace & 255)) {
      delete h;
      return fail(nullptr, PMG_ERR_OOM, "workspace too small or not 256-byte aligned");
    }
    h->ws = workspace;
  } else {
    cudaError_t e = cudaMalloc(&h->ws, pl.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return fail(nullptr, PMG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->ws_owned = true;
  }
  pl.carve((char *)h->ws);
  auto bail = [&](int code, const std::string &m) {
    if (h->ws_owned) cudaFree(h->ws);
    if (h->hred) cudaFreeHost(h->hred);
    if (h->hactive) cudaFreeHost(h->hactive);
    if (h->hctl) cudaFreeHost(h->hctl);
    delete h;
    return fail(nullptr, code, m);
  };
  if (cudaMallocHost(&h->hred, sizeof(unsigned long long) * 3 * h->P) != cudaSuccess ||
      cudaMallocHost(&h->hactive, sizeof(int) * h->P) != cudaSuccess ||
      cudaMallocHost(&h->hctl, sizeof(LoopCtl)) != cudaSuccess)
    return bail(PMG_ERR_OOM, "pinned host allocation failed");
  // zero everything: the pad columns of every grid function must stay zero
  cudaError_t e = cudaMemsetAsync(h->ws, 0, pl.total, h->stream);
  if (e != cudaSuccess) return bail(PMG_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  if (upload_minv(h) != PMG_OK) return bail(PMG_ERR_CUDA, h->err);
  if (h->opt.autotune) {
    MGCtx M = mgctx(h);
    if (autotune(M, 0, h->P, h->cf_sub[0]) != PMG_OK) return bail(PMG_ERR_CUDA, h->err);
  }
  if (h->groups > 1) {
    // the coarse chain runs single grids: it takes the narrow tuning of every level
    for (int l = 0; l < h->H.L; ++l) h->Hc.tune[l][0] = h->Hc.tune[l][1] = h->H.tune[l][1];
    int least = 0, greatest = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
              cudaStreamCreateWithPriority(&h->s_chain, cudaStreamNonBlocking, greatest) == cudaSuccess &&
              cudaStreamCreateWithPriority(&h->s_post, cudaStreamNonBlocking, least) == cudaSuccess &&
              cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&h->ev_chain_end, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&h->ev_post_end, cudaEventDisableTiming) == cudaSuccess;
    for (int g = 0; ok && g < h->groups; ++g)
      ok = cudaEventCreateWithFlags(&h->ev_fas[g], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&h->ev_chain[g], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      *out = h;  // let destroy release what was created
      pfasst_mg_destroy(h);
      *out = nullptr;
      return fail(nullptr, PMG_ERR_CUDA, "creating the pipeline streams failed");
    }
  }
  *out = h;
  return PMG_OK;
}

int pfasst_mg_set_initial(pmg_handle h, const double *u0, int on_device) {
  if (h && !h->kids.empty()) return fail(h, PMG_ERR_INVALID_ARG, "batch handle: use the pfasst_mg_batch_* calls");
  if (!h || !u0) return fail(h, PMG_ERR_INVALID_ARG, "null argument");
  const size_t N = (size_t)h->gf.nz * h->gf.ny * h->gf.n;
  const double *src = u0;
  if (!on_device) {
    PMG_CUDA(h, cudaMemcpyAsync(h->dense, u0, N * 8, cudaMemcpyHostToDevice, h->stream));
    src = h->dense;
  }
  PMG_CUDA(h, k_pack(h->L(), h->gf, src, 0, h->u0, 0, 1));
  PMG_RET(spread(h));
  if (!on_device) PMG_CUDA(h, cudaStreamSynchronize(h->stream));  // host buffer reusable on return
  return PMG_OK;
}

int pfasst_mg_predict(pmg_handle h) {
  if (h && !h->kids.empty()) return fail(h, PMG_ERR_INVALID_ARG, "batch handle: use the pfasst_mg_batch_* calls");
  if (!h) return fail(h, PMG_ERR_INVALID_ARG, "null handle");
  return predict(h);
}

int pfasst_mg_sweep(pmg_handle h, int level) {
  if (h && !h->kids.empty()) return fail(h, PMG_ERR_INVALID_ARG, "batch handle: use the pfasst_mg_batch_* calls");
  if (!h) return fail(h, PMG_ERR_INVALID_ARG, "null handle");
  h->spread_state = false;
  if (level == 0) {
    if (ffree(h) && !h->q_valid) PMG_RET(fine_residual(h));
    h->q_valid = false;
    return sweep(h, 0, 0, h->P);
  }
  if (level >= 1 && level == h->nlevels - 1) return coarse_chain(h);
  if (level == 1 && h->nlevels == 3) {
    // the iteration leaves F_1 stale after the level-2 correction: refresh it first
    PMG_CUDA(h, k_apply_A(h->L(), h->gc, h->nu, h->Uc, h->gc.slab, h->Fc, h->gc.slab, h->P * h->sc));
    return sweep(h, 1, 0, h->P);
  }
  return fail(h, PMG_ERR_INVALID_ARG, "level must be in [0, nlevels)");
}

int pfasst_mg_iterate(pmg_handle h, int max_iter, double tol, int *iters_done, double *final_res) {
  if (h && !h->kids.empty()) return fail(h, PMG_ERR_INVALID_ARG, "batch handle: use the pfasst_mg_batch_* calls");
  if (!h || max_iter < 0) return fail(h, PMG_ERR_INVALID_ARG, "bad argument");
  if (iters_done) *iters_done = 0;
  if (!h->predicted) PMG_RET(predict(h));
  double res = INFINITY;
  if (max_iter > 0 && device_loop_ok(h)) {
    if (ffree(h) && !h->q_valid) PMG_RET(fine_residual(h));  // after a standalone sweep
    int k = 0;
    PMG_RET(run_device_loop(h, max_iter, tol, &k, &res));
    h->q_valid = ffree(h);
    if (sweep_timeouts()) return fail(h, PMG_ERR_TIMEOUT, "a TMA-staged sweep timed out waiting for its loads");
    if (interp_timeouts())
      return fail(h, PMG_ERR_TIMEOUT, "the TMA-staged interpolation timed out waiting for its loads");
    if (coop_timeouts()) return fail(h, PMG_ERR_TIMEOUT, "a grid barrier of the persistent V-cycle timed out");
    if (iters_done) *iters_done = k;
    if (final_res) *final_res = res;
    if (std::isnan(res) || std::isinf(res)) return fail(h, PMG_ERR_DIVERGED, "collocation residual is NaN/Inf");
    return res <= tol ? PMG_OK : PMG_NOT_CONVERGED;
  }
  for (int k = 0; k < max_iter; ++k) {
    if (ffree(h) && !h->q_valid) PMG_RET(fine_residual(h));  // after a standalone sweep
    if (use_graphs(h)) PMG_RET(run_graph(h, h->g_iter, iteration));
    else PMG_RET(iteration(h));
    h->q_valid = ffree(h);
    PMG_CUDA(h, cudaStreamSynchronize(h->stream));
    if (sweep_timeouts()) return fail(h, PMG_ERR_TIMEOUT, "a TMA-staged sweep timed out waiting for its loads");
    if (interp_timeouts())
      return fail(h, PMG_ERR_TIMEOUT, "the TMA-staged interpolation timed out waiting for its loads");
    if (coop_timeouts()) return fail(h, PMG_ERR_TIMEOUT, "a grid barrier of the persistent V-cycle timed out");
    if (!h->g_iter.recs.empty() && use_graphs(h)) PMG_RET(harvest(h, h->g_iter));
    res = 0.0;
    for (int p = 0; p < h->P; ++p) {
      const double r = bits_to_double(h->hred[2 * h->P + p]);
      if (!(r <= res)) res = r;
    }
    if (iters_done) *iters_done = k + 1;
    if (final_res) *final_res = res;
    if (std::isnan(res) || std::isinf(res)) return fail(h, PMG_ERR_DIVERGED, "collocation residual is NaN/Inf");
    if (res <= tol) return PMG_OK;
  }
  return PMG_NOT_CONVERGED;
}

int pfasst_mg_residual(pmg_handle h, double *res) {
  if (h && !h->kids.empty()) return fail(h, PMG_ERR_INVALID_ARG, "batch handle: use the pfasst_mg_batch_* calls");
  if (!h || !res) return fail(h, PMG_ERR_INVALID_ARG, "null argument");
  PMG_RET(fine_residual(h));
  h->q_valid = ffree(h);
  PMG_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int p = 0; p < h->P; ++p) res[p] = bits_to_double(h->hred[2 * h->P + p]);
  return PMG_OK;
}

int pfasst_mg_get_solution(pmg_handle h, int slice, int node, double *out, int on_device) {
  if (h && !h->kids.empty()) return fail(h, PMG_ERR_INVALID_ARG, "batch handle: use the pfasst_mg_batch_* calls");
  if (!h || !out || slice < 0 || slice >= h->P || node < 0 || node >= h->sf)
    return fail(h, PMG_ERR_INVALID_ARG, "bad argument");
  const size_t N = (size_t)h->gf.nz * h->gf.ny * h->gf.n;
  const double *src = h->Uf + ((long long)slice * h->sf + node) * h->gf.slab;
  double *dst = on_device ? out : h->dense;
  PMG_CUDA(h, k_unpack(h->L(), h->gf, src, 0, dst, 0, 1));
  if (!on_device) PMG_CUDA(h, cudaMemcpyAsync(out, h->dense, N * 8, cudaMemcpyDeviceToHost, h->stream));
  PMG_CUDA(h, cudaStreamSynchronize(h->stream));
  return PMG_OK;
}

int pfasst_mg_get_state(pmg_handle h, int level, double *out) {
  if (h && !h->kids.empty()) return fail(h, PMG_ERR_INVALID_ARG, "batch handle: use the pfasst_mg_batch_* calls");
  if (!h || !out || level < 0 || level >= h->nlevels) return fail(h, PMG_ERR_INVALID_ARG, "bad argument");
  const LevelRef v = level_ref(h, level);
  const Grid &g = *v.g;
  const int s = v.s;
  const double *U = v.U;
  const size_t N = (size_t)g.nz * g.ny * g.n;
  for (int p = 0; p < h->P; ++p)
    for (int m = 0; m < s; ++m) {
      PMG_CUDA(h, k_unpack(h->L(), g, U + ((long long)p * s + m) * g.slab, 0, h->dense, 0, 1));
      PMG_CUDA(h, cudaMemcpyAsync(out + ((size_t)p * s + m) * N, h->dense, N * 8, cudaMemcpyDeviceToHost, h->stream));
      PMG_CUDA(h, cudaStreamSynchronize(h->stream));
    }
  return PMG_OK;
}

int pfasst_mg_advance(pmg_handle h) {
  if (h && !h->kids.empty()) return fail(h, PMG_ERR_INVALID_ARG, "batch handle: use the pfasst_mg_batch_* calls");
  if (!h) return fail(h, PMG_ERR_INVALID_ARG, "null handle");
  const long long last = ((long long)(h->P - 1) * h->sf + (h->sf - 1)) * h->gf.slab;
  PMG_CUDA(h, k_copy(h->L(), h->gf, h->Uf + last, 0, h->u0, 0, 1));
  return spread(h);
}

long long pfasst_mg_launch_count(pmg_handle h) { return h ? h->launches : -1; }

int pfasst_mg_tuning(pmg_handle h, int level, int narrow, int *fused, int *param, int *threads) {
  if (!h || !h->kids.empty() || level < 0 || level >= h->H.L || !fused || !param || !threads)
    return fail(h, PMG_ERR_INVALID_ARG, "bad argument");
  const Tune &t = h->H.tune[level][narrow ? 1 : 0];
  *fused = t.fused;
  *param = t.param;
  *threads = t.threads;
  return PMG_OK;
}

int pfasst_mg_set_tuning(pmg_handle h, int level, int narrow, int fused, int param, int threads) {
  if (!h || !h->kids.empty() || level < 0 || level >= h->H.L - 1 || fused < 0 || fused > 3)
    return fail(h, PMG_ERR_INVALID_ARG, "bad argument");
  const Grid &g = h->H.lev[level];
  Tune t{fused, param, threads};
  if (fused == 0 && (param < 32 || param > 1024 || param % 32)) return fail(h, PMG_ERR_INVALID_ARG, "threads per block");
  if (fused >= 1) {
    if (h->opt.smoother != PMG_SMOOTHER_RBGS || g.dim != 3 || g.n < 15 || param < 0 || param > g.n)
      return fail(h, PMG_ERR_UNSUPPORTED, "the fused sweep needs 3D red-black Gauss-Seidel, n >= 15, 0 <= z chunk <= n");
    if (g.order == 4) return fail(h, PMG_ERR_UNSUPPORTED, "the fused sweeps run the second-order stencil only");
    if (fused == 1 && threads != 256 && !(threads == 512 && g.pitch >= 128))
      return fail(h, PMG_ERR_INVALID_ARG, "fused sweep threads: 256, or 512 for rows of >= 128");
    if (fused >= 2 && !rbgs_tma_supported(g, h->H.pr))
      return fail(h, PMG_ERR_UNSUPPORTED, "the TMA-staged sweep needs FP32 (mixed precision) and n = 127 or 255");
    if (fused >= 2) t.threads = rbgs_tma_threads(g, fused == 3);
  }
  PMG_CUDA(h, cudaStreamSynchronize(h->stream));
  drop_graph(h->g_pred);
  drop_graph(h->g_pred_spread);
  drop_graph(h->g_iter);
  drop_graph(h->g_loop);
  h->H.tune[level][narrow ? 1 : 0] = t;
  if (h->groups > 1 && narrow) h->Hc.tune[level][0] = h->Hc.tune[level][1] = t;
  return PMG_OK;
}

int pfasst_mg_profile(pmg_handle h, int enable, long long min_points) {
  if (!h || min_points < 0) return fail(h, PMG_ERR_INVALID_ARG, "bad argument");
  h->prof.on = enable != 0;
  h->prof.min_points = min_points;
  return PMG_OK;
}

}  // extern "C"

namespace {

// resolve the pending event pairs of a profiler and aggregate per (kernel, n, precision)
cudaError_t prof_aggregate(Profiler &P, pmg_kernel_stat *out, int capacity, int *count) {
  for (const ProfRec &r : P.recs) {
    float ms = 0.f;
    cudaError_t e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) return e;
    P.done.push_back(ProfDone{r.kid, r.n, r.prec, r.pts, ms});
  }
  P.recs.clear();
  P.used = 0;
  std::vector<pmg_kernel_stat> agg;
  for (const ProfDone &r : P.done) {
    size_t q = 0;
    for (; q < agg.size(); ++q)
      if (agg[q].kernel == r.kid && agg[q].n == r.n && agg[q].precision == r.prec) break;
    if (q == agg.size()) agg.push_back(pmg_kernel_stat{r.kid, r.n, r.prec, 0, 0, 0.0});
    agg[q].launches += 1;
    agg[q].points += r.pts;
    agg[q].ms += r.ms;
  }
  P.done.clear();
  *count = (int)agg.size();
  for (int q = 0; q < capacity && q < (int)agg.size(); ++q) out[q] = agg[q];
  return cudaSuccess;
}

}  // namespace

extern "C" {

int pfasst_mg_profile_read(pmg_handle h, pmg_kernel_stat *out, int capacity, int *count) {
  if (!h || !count || capacity < 0 || (capacity > 0 && !out)) return fail(h, PMG_ERR_INVALID_ARG, "bad argument");
  PMG_CUDA(h, cudaStreamSynchronize(h->stream));
  PMG_CUDA(h, prof_aggregate(h->prof, out, capacity, count));
  return PMG_OK;
}

const char *pfasst_mg_kernel_name(int kernel) {
  static const char *names[K_COUNT] = {"residual0", "smooth_jacobi", "smooth_rbgs", "residual_restrict",
                                       "prolong_add", "coarse_solve", "update_u", "zero", "apply_A", "sf_rhs",
                                       "fas_restrict", "interp_space", "colloc_residual", "copy", "pack",
                                       "unpack", "interp_time", "rbgs_sweep3d", "resrestrict3d", "prolong3d",
                                       "resid_pt", "fine_rhs_residual", "rbgs_sweep3d_zero",
                                       "rbgs_sweep3d_upd", "net_resid", "net_layer1", "net_layer2_mma",
                                       "net_layer3", "net_loss", "net_layer3_bwd", "net_layer2_mma_bwd",
                                       "net_wgrad", "net_adam", "net_sample", "vcycle_tail", "vcycle_coop"};
  return kernel >= 0 && kernel < K_COUNT ? names[kernel] : "unknown";
}

int pfasst_mg_destroy(pmg_handle h) {
  if (!h) return PMG_OK;
  if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
  for (pmg_ctx *k : h->kids) {
    drop_graph(k->g_pred);
    drop_graph(k->g_pred_spread);
    drop_graph(k->g_iter);
    drop_graph(k->g_loop);
    if (k->hred) cudaFreeHost(k->hred);
    if (k->hactive) cudaFreeHost(k->hactive);
    delete k;
  }
  for (cudaStream_t b : h->branch) cudaStreamDestroy(b);
  for (cudaEvent_t e : h->join) cudaEventDestroy(e);
  if (h->fork) cudaEventDestroy(h->fork);
  if (h->bexec) cudaGraphExecDestroy(h->bexec);
  drop_graph(h->g_pred);
  drop_graph(h->g_pred_spread);
  drop_graph(h->g_iter);
  drop_graph(h->g_loop);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->s_chain) cudaStreamDestroy(h->s_chain);
  if (h->s_post) cudaStreamDestroy(h->s_post);
  for (cudaEvent_t e : {h->ev_fork, h->ev_chain_end, h->ev_post_end})
    if (e) cudaEventDestroy(e);
  for (int g = 0; g < kMaxGroups; ++g) {
    if (h->ev_fas[g]) cudaEventDestroy(h->ev_fas[g]);
    if (h->ev_chain[g]) cudaEventDestroy(h->ev_chain[g]);
  }
  if (h->net) {
    if (h->net->mem) cudaFree(h->net->mem);
    delete h->net;
  }
  if (h->ws_owned && h->ws) cudaFree(h->ws);
  if (h->hred) cudaFreeHost(h->hred);
  if (h->hactive) cudaFreeHost(h->hactive);
  if (h->hctl) cudaFreeHost(h->hctl);
  delete h;
  return PMG_OK;
}

const char *pfasst_mg_last_error(pmg_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int pfasst_mg_check_narrowing(long long samples, unsigned long long seed, long long *mismatches) {
  if (samples < 0 || !mismatches) return fail(nullptr, PMG_ERR_INVALID_ARG, "bad argument");
  unsigned long long *bad = nullptr, hbad = 0;
  if (cudaMalloc(&bad, sizeof bad[0]) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, PMG_ERR_CUDA, "cudaMalloc failed");
  }
  cudaError_t e = cudaMemset(bad, 0, sizeof bad[0]);
  if (e == cudaSuccess) e = k_narrow_check(nullptr, samples, seed, bad);
  if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost);
  cudaFree(bad);
  if (e != cudaSuccess) return fail(nullptr, PMG_ERR_CUDA, std::string("narrowing check: ") + cudaGetErrorString(e));
  *mismatches = (long long)hbad;
  return PMG_OK;
}

int pfasst_mg_check_widening(long long *mismatches) {
  if (!mismatches) return fail(nullptr, PMG_ERR_INVALID_ARG, "bad argument");
  unsigned long long *bad = nullptr, hbad = 0;
  if (cudaMalloc(&bad, sizeof bad[0]) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, PMG_ERR_CUDA, "cudaMalloc failed");
  }
  cudaError_t e = cudaMemset(bad, 0, sizeof bad[0]);
  if (e == cudaSuccess) e = k_widen_check(nullptr, bad);
  if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost);
  cudaFree(bad);
  if (e != cudaSuccess) return fail(nullptr, PMG_ERR_CUDA, std::string("widening check: ") + cudaGetErrorString(e));
  *mismatches = (long long)hbad;
  return PMG_OK;
}

int pfasst_mg_helmholtz_solve(const pmg_grid *grid, double c, int batch, const double *b, double *u,
                              const pmg_options *opt, void *stream, int *cycles_done) {
  pmg_nodes_desc fn{3, 0};
  pmg_levels lv{1, {0, 0}};
  std::string why;
  int rc = validate(grid, &fn, &lv, batch < 1 ? 1 : batch, opt, why);
  if (rc != PMG_OK) return fail(nullptr, rc, why);
  if (batch < 1 || !b || !u || !(c >= 0) || !std::isfinite(c)) return fail(nullptr, PMG_ERR_INVALID_ARG, "bad argument");
  pmg_options o;
  if (opt) o = *opt; else pfasst_mg_default_options(&o);
  cudaStream_t st = (cudaStream_t)stream;
  Grid g = make_grid(grid->dim, grid->n, grid_order(grid));
  Hier H;
  Plan pl;
  double *bp = nullptr, *up = nullptr;
  void *minv = nullptr;
  unsigned long long *red = nullptr;
  int *active = nullptr;
  pl.add((void **)&bp, (size_t)g.slab * batch * 8);
  pl.add((void **)&up, (size_t)g.slab * batch * 8);
  plan_hier(pl, H, grid->dim, grid->n, batch, o.precision == PMG_PREC_MIXED ? F32 : F64, o.smoother, 0,
            grid_order(grid));
  const int n3 = grid->dim == 1 ? 3 : (grid->dim == 2 ? 9 : 27);
  pl.add(&minv, (size_t)n3 * n3 * H.tsize);
  pl.add((void **)&red, sizeof(unsigned long long) * 2 * batch);
  pl.add((void **)&active, sizeof(int) * batch);
  void *block = nullptr;
  if (cudaMallocAsync(&block, pl.total, st) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, PMG_ERR_OOM, "cudaMallocAsync failed");
  }
  pl.carve((char *)block);
  unsigned long long *hred = nullptr;
  int *hactive = nullptr;
  int result = PMG_OK;
  long long launches = 0;
  do {
    if (cudaMallocHost(&hred, sizeof(unsigned long long) * 2 * batch) != cudaSuccess ||
        cudaMallocHost(&hactive, sizeof(int) * batch) != cudaSuccess) {
      result = fail(nullptr, PMG_ERR_OOM, "pinned host allocation failed");
      break;
    }
    std::vector<double> M;
    coarsest_inverse(grid->dim, c, M);
    std::vector<char> buf(M.size() * H.tsize);
    for (size_t q = 0; q < M.size(); ++q) {
      if (H.tsize == 8) std::memcpy(buf.data() + q * 8, &M[q], 8);
      else { float fv = (float)M[q]; std::memcpy(buf.data() + q * 4, &fv, 4); }
    }
    Launch Ln{st, &launches, nullptr};
    if (cudaMemsetAsync(block, 0, pl.total, st) != cudaSuccess ||
        cudaMemcpyAsync(minv, buf.data(), buf.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        k_pack(Ln, g, b, (long long)g.nz * g.ny * g.n, bp, g.slab, batch) != cudaSuccess ||
        k_pack(Ln, g, u, (long long)g.nz * g.ny * g.n, up, g.slab, batch) != cudaSuccess) {
      result = fail(nullptr, PMG_ERR_CUDA, "set-up copy failed");
      break;
    }
    MGCtx Mc{Ln, &H, &o, red, active, hred, hactive, nullptr, st};
    int cyc = 0;
    result = solve_substep(Mc, 0, batch, c, minv, bp, g.slab, nullptr, 0, up, g.slab, &cyc);
    if (result != PMG_OK) break;
    if (k_unpack(Ln, g, up, g.slab, u, (long long)g.nz * g.ny * g.n, batch) != cudaSuccess) {
      result = fail(nullptr, PMG_ERR_CUDA, "unpack failed");
      break;
    }
    if (cycles_done) *cycles_done = cyc;
  } while (0);
  cudaFreeAsync(block, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (hred) cudaFreeHost(hred);
  if (hactive) cudaFreeHost(hactive);
  if (result == PMG_OK && e != cudaSuccess) result = fail(nullptr, PMG_ERR_CUDA, cudaGetErrorString(e));
  if (result == PMG_OK && coop_timeouts())
    result = fail(nullptr, PMG_ERR_TIMEOUT, "a grid barrier of the persistent V-cycle timed out");
  return result;
}

}  // extern "C"

// ----------------------------------------------------------------- uneven batch
//
// Independent heat problems of different grids, node counts, nu and dt: each is a
// single-level SDC solver (one time slice) with its own multigrid hierarchy carved
// from one workspace.  A time step of every problem -- right-hand sides, `sweeps` SDC
// sweeps, residual, advance to the step's end value -- is captured once into a CUDA
// graph in which every problem is its own branch, so the small problems fill the GPU
// side by side; the graph is replayed once per time step.

namespace {

int validate_problem(const pmg_problem_desc &d, const pmg_options *o, std::string &why) {
  pmg_nodes_desc fn{d.nodes, 0};
  pmg_levels lv{1, {0, 0}};
  int rc = validate(&d.grid, &fn, &lv, 1, o, why);
  if (rc != PMG_OK) return rc;
  if (!(d.nu > 0) || !(d.dt > 0) || !std::isfinite(d.nu) || !std::isfinite(d.dt)) {
    why = "nu and dt must be positive and finite";
    return PMG_ERR_INVALID_ARG;
  }
  return PMG_OK;
}

pmg_ctx *make_kid(const pmg_problem_desc &d, const pmg_options &o) {
  pmg_nodes_desc fn{d.nodes, 0};
  pmg_levels lv{1, {0, 0}};
  // the problems of a batch run side by side on graph branches: a persistent V-cycle
  // that holds every SM would serialise them, so they keep the per-level launches
  pmg_options ko = o;
  ko.single_grid_vcycle = 0;
  return make_ctx(&d.grid, &fn, &lv, d.nu, d.dt, 1, &ko);
}

// one time step of one problem (captured into the batch graph)
int batch_step_body(pmg_ctx *k, int sweeps) {
  PMG_RET(fine_residual(k));
  for (int i = 0; i < sweeps; ++i) PMG_RET(iteration(k));
  const long long last = (long long)(k->sf - 1) * k->gf.slab;
  PMG_CUDA(k, k_copy(k->L(), k->gf, k->Uf + last, 0, k->u0, 0, 1));
  return spread(k);
}

bool is_batch(const pmg_ctx *h) { return h && !h->kids.empty(); }

}  // namespace

extern "C" {

int pfasst_mg_batch_workspace_bytes(int nprob, const pmg_problem_desc *probs, const pmg_options *opt,
                                    size_t *bytes) {
  if (nprob < 1 || nprob > 4096 || !probs || !bytes) return fail(nullptr, PMG_ERR_INVALID_ARG, "bad argument");
  pmg_options o;
  if (opt) o = *opt; else pfasst_mg_default_options(&o);
  if (o.vcycles < 1) return fail(nullptr, PMG_ERR_UNSUPPORTED, "batches run a fixed number of V-cycles (vcycles >= 1)");
  size_t total = 0;
  for (int i = 0; i < nprob; ++i) {
    std::string why;
    int rc = validate_problem(probs[i], &o, why);
    if (rc != PMG_OK) return fail(nullptr, rc, "problem " + std::to_string(i) + ": " + why);
    pmg_ctx *k = make_kid(probs[i], o);
    if (!k) return fail(nullptr, PMG_ERR_OOM, "host allocation failed");
    Plan pl;
    plan_ctx(pl, k);
    total += pl.total;
    delete k;
  }
  *bytes = total;
  return PMG_OK;
}

int pfasst_mg_create_batch(int nprob, const pmg_problem_desc *probs, const pmg_options *opt, void *stream,
                           void *workspace, size_t workspace_bytes, pmg_handle *out) {
  if (!out) return fail(nullptr, PMG_ERR_INVALID_ARG, "out is null");
  *out = nullptr;
  size_t need = 0;
  int rc = pfasst_mg_batch_workspace_bytes(nprob, probs, opt, &need);
  if (rc != PMG_OK) return rc;
  pmg_options o;
  if (opt) o = *opt; else pfasst_mg_default_options(&o);
  pmg_ctx *h = new (std::nothrow) pmg_ctx();
  if (!h) return fail(nullptr, PMG_ERR_OOM, "host allocation failed");
  h->opt = o;
  h->stream = (cudaStream_t)stream;
  if (workspace) {
    if (workspace_bytes < need || ((uintptr_t)workspace & 255)) {
      delete h;
      return fail(nullptr, PMG_ERR_OOM, "workspace too small or not 256-byte aligned");
    }
    h->ws = workspace;
  } else {
    cudaError_t e = cudaMalloc(&h->ws, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return fail(nullptr, PMG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    h->ws_owned = true;
  }
  std::string why;
  char *base = (char *)h->ws;
  rc = PMG_OK;
  for (int i = 0; i < nprob && rc == PMG_OK; ++i) {
    pmg_ctx *k = make_kid(probs[i], o);
    if (!k) { rc = PMG_ERR_OOM; why = "host allocation failed"; break; }
    h->kids.push_back(k);
    k->stream = h->stream;
    fill_coefficients(k);
    Plan pl;
    plan_ctx(pl, k);
    pl.carve(base);
    base += pl.total;
    if (cudaMallocHost(&k->hred, sizeof(unsigned long long) * 3) != cudaSuccess ||
        cudaMallocHost(&k->hactive, sizeof(int)) != cudaSuccess) {
      rc = PMG_ERR_OOM;
      why = "pinned host allocation failed";
      break;
    }
    if (cudaMemsetAsync(k->ws ? k->ws : (void *)(base - pl.total), 0, pl.total, h->stream) != cudaSuccess ||
        upload_minv(k) != PMG_OK) {
      rc = PMG_ERR_CUDA;
      why = "set-up of problem " + std::to_string(i) + " failed";
      break;
    }
    if (o.autotune) {
      MGCtx M = mgctx(k);
      if (autotune(M, 0, 1, k->cf_sub[0]) != PMG_OK) { rc = PMG_ERR_CUDA; why = k->err; break; }
    }
  }
  if (rc == PMG_OK) {
    const int nb = nprob < 32 ? nprob : 32;
    h->branch.resize(nb, nullptr);
    h->join.resize(nb, nullptr);
    for (int b = 0; b < nb && rc == PMG_OK; ++b)
      if (cudaStreamCreateWithFlags(&h->branch[b], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->join[b], cudaEventDisableTiming) != cudaSuccess) {
        rc = PMG_ERR_CUDA;
        why = "stream creation failed";
      }
    if (rc == PMG_OK && cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) != cudaSuccess) {
      rc = PMG_ERR_CUDA;
      why = "event creation failed";
    }
  }
  if (rc != PMG_OK) {
    std::string msg = why;
    pfasst_mg_destroy(h);
    return fail(nullptr, rc, msg);
  }
  *out = h;
  return PMG_OK;
}

int pfasst_mg_batch_set_initial(pmg_handle h, int prob, const double *u0, int on_device) {
  if (!is_batch(h) || prob < 0 || prob >= (int)h->kids.size()) return fail(h, PMG_ERR_INVALID_ARG, "bad argument");
  int rc = pfasst_mg_set_initial(h->kids[prob], u0, on_device);
  if (rc != PMG_OK) return fail(h, rc, h->kids[prob]->err);
  return PMG_OK;
}

int pfasst_mg_batch_run(pmg_handle h, int steps, int sweeps, double *residuals) {
  if (!is_batch(h) || steps < 0 || sweeps < 1) return fail(h, PMG_ERR_INVALID_ARG, "bad argument");
  const int np = (int)h->kids.size(), nb = (int)h->branch.size();
  if (!h->opt.use_graphs) {  // eager: the problems one after the other on the handle's stream
    for (int st = 0; st < steps; ++st)
      for (pmg_ctx *k : h->kids) {
        const long long before = k->launches;
        int rc = batch_step_body(k, sweeps);
        h->launches += k->launches - before;
        if (rc != PMG_OK) return fail(h, rc, k->err);
      }
  } else {
    if (h->bexec && h->bsweeps != sweeps) {
      cudaGraphExecDestroy(h->bexec);
      h->bexec = nullptr;
    }
    if (!h->bexec) {
      if (!h->cap_stream) PMG_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
      PMG_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
      int rc = cudaEventRecord(h->fork, h->cap_stream) == cudaSuccess ? PMG_OK : PMG_ERR_CUDA;
      for (int b = 0; b < nb && rc == PMG_OK; ++b)
        if (cudaStreamWaitEvent(h->branch[b], h->fork, 0) != cudaSuccess) rc = PMG_ERR_CUDA;
      long long kernels = 0;
      std::string why;
      for (int i = 0; i < np && rc == PMG_OK; ++i) {
        pmg_ctx *k = h->kids[i];
        const long long before = k->launches;
        k->stream = h->branch[i % nb];
        rc = batch_step_body(k, sweeps);
        k->stream = h->stream;
        kernels += k->launches - before;
        k->launches = before;
        if (rc != PMG_OK) why = k->err;
      }
      for (int b = 0; b < nb && rc == PMG_OK; ++b)
        if (cudaEventRecord(h->join[b], h->branch[b]) != cudaSuccess ||
            cudaStreamWaitEvent(h->cap_stream, h->join[b], 0) != cudaSuccess)
          rc = PMG_ERR_CUDA;
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
      if (rc != PMG_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(h, rc != PMG_OK ? rc : PMG_ERR_CUDA,
                    "batch capture failed: " + (why.empty() ? std::string(cudaGetErrorString(e)) : why));
      }
      e = cudaGraphInstantiate(&h->bexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        h->bexec = nullptr;
        return fail(h, PMG_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
      }
      h->bsweeps = sweeps;
      h->bkernels = kernels;
    }
    for (int st = 0; st < steps; ++st) {
      PMG_CUDA(h, cudaGraphLaunch(h->bexec, h->stream));
      h->launches += h->bkernels;
    }
  }
  PMG_CUDA(h, cudaStreamSynchronize(h->stream));
  if (residuals)
    for (int i = 0; i < np; ++i) residuals[i] = bits_to_double(h->kids[i]->hred[2]);
  return PMG_OK;
}

int pfasst_mg_batch_get_solution(pmg_handle h, int prob, double *out, int on_device) {
  if (!is_batch(h) || !out || prob < 0 || prob >= (int)h->kids.size())
    return fail(h, PMG_ERR_INVALID_ARG, "bad argument");
  pmg_ctx *k = h->kids[prob];
  const size_t N = (size_t)k->gf.nz * k->gf.ny * k->gf.n;
  double *dst = on_device ? out : k->dense;
  PMG_CUDA(h, k_unpack(k->L(), k->gf, k->u0, 0, dst, 0, 1));
  if (!on_device) PMG_CUDA(h, cudaMemcpyAsync(out, k->dense, N * 8, cudaMemcpyDeviceToHost, k->stream));
  PMG_CUDA(h, cudaStreamSynchronize(k->stream));
  return PMG_OK;
}

}  // extern "C"

// ----------------------------------------------------------------- learned correction network
//
// Training: a pmg_net handle owns the parameters, the Adam moments and the scratch of
// the forward / backward kernels for a batch of n^3 grids.  Deployment:
// pfasst_mg_set_smoother_net copies a parameter vector into a PFASST handle, where it
// replaces the second pre-smoothing sweep on the chosen multigrid levels; levels on
// which the measured V-cycle contraction does not improve keep the plain sweep.

struct pmg_net {
  int batch = 0, n = 0;
  cudaStream_t stream = nullptr;
  void *mem = nullptr;
  float *prm = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *xs = nullptr, *ts = nullptr;
  double *loss = nullptr;
  double *u64 = nullptr, *zero64 = nullptr;  // multigrid-shaped samples (FP64, dense)
  unsigned long long *mx = nullptr;
  NetScratch s;
  int step = 0;
  long long launches = 0;
  Profiler prof;
  std::string err;
  Launch L() { return Launch{stream, &launches, &prof}; }
  NetGrid grid() const { return NetGrid{batch, n, n, (long long)n * n * n}; }
  size_t pts() const { return (size_t)batch * n * n * n; }
};

namespace {

int nfail(pmg_net *h, int code, const std::string &msg) {
  if (h) h->err = msg; else g_create_error = msg;
  return code;
}

#define PMG_NCUDA(h, expr)                                                                 \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return nfail(h, PMG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));   \
  } while (0)

cudaMemcpyKind kind_in(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

// V-cycle contraction on the fine level of h with the handle's current network
// settings: from uniform noise e with f = 0, rho = (|e_4| / |e_1|)^(1/3) in the max
// norm after V-cycles 1 and 4, worst over the fine sub-step operators
int net_measure(pmg_ctx *h, double *rho) {
  MGCtx M = mgctx(h);
  Hier &H = h->H;
  const Grid &g = H.lev[0];
  double worst = 0.0;
  for (int m = 0; m < h->sf - 1; ++m) {
    PMG_CUDA(h, k_net_noise(h->L(), g, H.pr, H.e[0], 1, 0x5eedULL + (unsigned long long)m));
    PMG_CUDA(h, cudaMemsetAsync(H.f[0], 0, (size_t)g.slab * H.tsize, h->stream));
    void *e = H.e[0];
    double nrm[2] = {0.0, 0.0};
    for (int k = 0; k < 4; ++k) {
      PMG_RET(vcycle(M, 0, 1, h->cf_sub[m], h->minv_slot(m), e, &e));
      if (k != 0 && k != 3) continue;
      PMG_CUDA(h, cudaMemsetAsync(h->red, 0, sizeof(unsigned long long), h->stream));
      PMG_CUDA(h, k_net_maxabs(h->L(), g, H.pr, e, 1, h->red));
      PMG_CUDA(h, cudaMemcpyAsync(h->hred, h->red, sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream));
      PMG_CUDA(h, cudaStreamSynchronize(h->stream));
      std::memcpy(&nrm[k == 3], h->hred, 8);
    }
    if (!std::isfinite(nrm[0]) || !std::isfinite(nrm[1])) { worst = INFINITY; break; }
    const double r = nrm[0] > 0.0 ? std::pow(nrm[1] / nrm[0], 1.0 / 3.0) : 0.0;
    worst = r > worst ? r : worst;
  }
  for (int l = 0; l < H.L; ++l) {
    const size_t bytes = (size_t)H.lev[l].slab * H.batch * H.tsize;
    PMG_CUDA(h, cudaMemsetAsync(H.e[l], 0, bytes, h->stream));
    if (H.e2[l]) PMG_CUDA(h, cudaMemsetAsync(H.e2[l], 0, bytes, h->stream));
  }
  PMG_CUDA(h, cudaMemsetAsync(H.f[0], 0, (size_t)g.slab * H.batch * H.tsize, h->stream));
  PMG_CUDA(h, cudaStreamSynchronize(h->stream));
  *rho = worst;
  return PMG_OK;
}

// one batch of training pairs into h->xs, h->ts, h->s.kappa: vmax = 0, smoothed noise;
// vmax > 0, grid b first gets k_b in 0..vmax V-cycles of (I - c_b Lap) u = 0 from
// noise (c_b from kappa_b), so the errors have the spectrum the multigrid iteration
// leaves, normalised to max 1
int net_draw(pmg_net *h, unsigned long long seed, double klo, double khi, int vmax) {
  const NetGrid g = h->grid();
  if (vmax == 0) {
    PMG_NCUDA(h, k_net_sample(h->L(), g, seed, (float)klo, (float)khi, h->xs, h->ts, h->s.kappa));
    return PMG_OK;
  }
  std::vector<float> kap(h->batch);
  for (int b = 0; b < h->batch; ++b) kap[b] = net_sample_kappa(seed, (float)klo, (float)khi, b);
  PMG_NCUDA(h, cudaMemcpyAsync(h->s.kappa, kap.data(), sizeof(float) * h->batch, cudaMemcpyHostToDevice, h->stream));
  PMG_NCUDA(h, k_net_sample_noise64(h->L(), g, seed, h->u64));
  pmg_options o;
  pfasst_mg_default_options(&o);
  o.smoother = PMG_SMOOTHER_RBGS;
  o.omega = 1.0;
  o.use_graphs = 0;
  o.autotune = 0;
  const pmg_grid grid{3, h->n};
  const double ih2 = (double)(h->n + 1) * (h->n + 1);
  for (int b = 0; b < h->batch; ++b) {
    o.vcycles = net_sample_vcycles(seed, vmax, b);
    if (o.vcycles == 0) continue;
    const double k = kap[b] < 1.0 / 6.0 - 1e-6 ? kap[b] : 1.0 / 6.0 - 1e-6;
    const double c = k / ((1.0 - 6.0 * k) * ih2);  // kappa = (c/h^2) / (1 + 6 c/h^2)
    const size_t off = (size_t)b * h->n * h->n * h->n;
    const int rc = pfasst_mg_helmholtz_solve(&grid, c, 1, h->zero64 + off, h->u64 + off, &o, h->stream, nullptr);
    if (rc != PMG_OK) return nfail(h, rc, std::string("sample V-cycles: ") + pfasst_mg_last_error(nullptr));
  }
  PMG_NCUDA(h, k_net_sample_finish(h->L(), g, h->u64, h->mx, h->xs, h->ts, h->s.kappa));
  return PMG_OK;
}

int check_sample_args(pmg_net *h, double kappa_lo, double kappa_hi, int vmax) {
  if (!(kappa_lo >= 0.0 && kappa_hi >= kappa_lo && kappa_hi <= 1.0 / 6.0))
    return nfail(h, PMG_ERR_INVALID_ARG, "need 0 <= kappa_lo <= kappa_hi <= 1/6");
  if (vmax < 0 || vmax > 8) return nfail(h, PMG_ERR_INVALID_ARG, "vcycles_max must be 0..8");
  if (vmax > 0 && (h->n < 7 || ((h->n + 1) & h->n) != 0))
    return nfail(h, PMG_ERR_INVALID_ARG, "multigrid-shaped samples need n = 2^p - 1 >= 7");
  return PMG_OK;
}

}  // namespace

extern "C" {

int pfasst_mg_net_param_count(void) { return kNetParams; }

int pfasst_mg_net_init(float *params, unsigned long long seed) {
  if (!params) return nfail(nullptr, PMG_ERR_INVALID_ARG, "params is NULL");
  net_init_params(params, seed);
  return PMG_OK;
}

int pfasst_mg_net_create(int batch, int n, void *stream, pmg_net_handle *out) {
  if (!out) return nfail(nullptr, PMG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (batch < 1 || n < 3 || n > 255 || (long long)batch * n * n * n > (1LL << 28))
    return nfail(nullptr, PMG_ERR_INVALID_ARG, "need batch >= 1, 3 <= n <= 255 and batch * n^3 <= 2^28");
  pmg_net *h = new (std::nothrow) pmg_net();
  if (!h) return nfail(nullptr, PMG_ERR_OOM, "host allocation failed");
  h->batch = batch;
  h->n = n;
  h->stream = (cudaStream_t)stream;
  const size_t P = align256(kNetParams * sizeof(float)), X = align256(h->pts() * sizeof(float));
  const size_t X64 = align256(h->pts() * sizeof(double));
  const size_t bytes = 4 * P + 2 * X + 2 * X64 + align256(sizeof(double) * 4096) + align256(8 * (size_t)batch) +
                       net_train_bytes(batch, n);
  if (cudaMalloc(&h->mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return nfail(nullptr, PMG_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  char *p = (char *)h->mem;
  h->prm = (float *)p; p += P;
  h->grad = (float *)p; p += P;
  h->m = (float *)p; p += P;
  h->v = (float *)p; p += P;
  h->xs = (float *)p; p += X;
  h->ts = (float *)p; p += X;
  h->loss = (double *)p; p += align256(sizeof(double) * 4096);
  h->u64 = (double *)p; p += X64;
  h->zero64 = (double *)p; p += X64;
  h->mx = (unsigned long long *)p; p += align256(8 * (size_t)batch);
  h->s = net_train_carve(p, batch, n);
  if (cudaMemsetAsync(h->zero64, 0, h->pts() * sizeof(double), h->stream) != cudaSuccess) {
    cudaGetLastError();
    pfasst_mg_net_destroy(h);
    return nfail(nullptr, PMG_ERR_CUDA, "cudaMemsetAsync failed");
  }
  std::vector<float> init(kNetParams);
  net_init_params(init.data(), 5);
  int rc = pfasst_mg_net_set_params(h, init.data());
  if (rc != PMG_OK) {
    g_create_error = h->err;
    pfasst_mg_net_destroy(h);
    return rc;
  }
  *out = h;
  return PMG_OK;
}

int pfasst_mg_net_set_params(pmg_net_handle h, const float *params) {
  if (!h || !params) return nfail(h, PMG_ERR_INVALID_ARG, "null handle or params");
  PMG_NCUDA(h, cudaMemcpyAsync(h->prm, params, kNetParams * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  PMG_NCUDA(h, cudaMemsetAsync(h->m, 0, kNetParams * sizeof(float), h->stream));
  PMG_NCUDA(h, cudaMemsetAsync(h->v, 0, kNetParams * sizeof(float), h->stream));
  PMG_NCUDA(h, cudaStreamSynchronize(h->stream));
  h->step = 0;
  return PMG_OK;
}

int pfasst_mg_net_get_params(pmg_net_handle h, float *params) {
  if (!h || !params) return nfail(h, PMG_ERR_INVALID_ARG, "null handle or params");
  PMG_NCUDA(h, cudaMemcpyAsync(params, h->prm, kNetParams * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  PMG_NCUDA(h, cudaStreamSynchronize(h->stream));
  return PMG_OK;
}

int pfasst_mg_net_forward(pmg_net_handle h, const float *x, float *y, int on_device) {
  if (!h || !x || !y) return nfail(h, PMG_ERR_INVALID_ARG, "null handle or array");
  const size_t bytes = h->pts() * sizeof(float);
  PMG_NCUDA(h, cudaMemcpyAsync(h->xs, x, bytes, kind_in(on_device), h->stream));
  PMG_NCUDA(h, k_net_pack(h->L(), h->prm, h->s));
  PMG_NCUDA(h, k_net_forward(h->L(), h->grid(), h->xs, h->prm, h->s, h->s.y));
  PMG_NCUDA(h, cudaMemcpyAsync(y, h->s.y, bytes, kind_out(on_device), h->stream));
  PMG_NCUDA(h, cudaStreamSynchronize(h->stream));
  return PMG_OK;
}

int pfasst_mg_net_gradients(pmg_net_handle h, const float *x, const float *t, const float *kappa, int power,
                            int on_device, float *grad, double *loss) {
  if (!h || !x || !t || !kappa || !grad) return nfail(h, PMG_ERR_INVALID_ARG, "null handle or array");
  if (power < 0 || power > 3) return nfail(h, PMG_ERR_INVALID_ARG, "power must be 0..3");
  const size_t bytes = h->pts() * sizeof(float);
  PMG_NCUDA(h, cudaMemcpyAsync(h->xs, x, bytes, kind_in(on_device), h->stream));
  PMG_NCUDA(h, cudaMemcpyAsync(h->ts, t, bytes, kind_in(on_device), h->stream));
  PMG_NCUDA(h, cudaMemcpyAsync(h->s.kappa, kappa, h->batch * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  PMG_NCUDA(h, cudaMemsetAsync(h->grad, 0, kNetParams * sizeof(float), h->stream));
  PMG_NCUDA(h, cudaMemsetAsync(h->loss, 0, sizeof(double), h->stream));
  PMG_NCUDA(h, k_net_pack(h->L(), h->prm, h->s));
  PMG_NCUDA(h, k_net_grads(h->L(), h->grid(), h->xs, h->ts, h->s.kappa, power, h->prm, h->grad, h->s, h->loss));
  PMG_NCUDA(h, cudaMemcpyAsync(grad, h->grad, kNetParams * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  double l = 0.0;
  PMG_NCUDA(h, cudaMemcpyAsync(&l, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  PMG_NCUDA(h, cudaStreamSynchronize(h->stream));
  if (loss) *loss = l;
  return PMG_OK;
}

int pfasst_mg_net_substep_pairs(pmg_net_handle h, const double *u0, const float *kappa, float *x, float *t,
                                int on_device) {
  if (!h || !u0 || !kappa || !x || !t) return nfail(h, PMG_ERR_INVALID_ARG, "null handle or array");
  if (h->n < 7 || ((h->n + 1) & h->n) != 0) return nfail(h, PMG_ERR_INVALID_ARG, "sub-step pairs need n = 2^p - 1 >= 7");
  for (int b = 0; b < h->batch; ++b)
    if (!(kappa[b] >= 0.0f && kappa[b] < 1.0f / 6.0f)) return nfail(h, PMG_ERR_INVALID_ARG, "need 0 <= kappa < 1/6");
  const NetGrid g = h->grid();
  const size_t n3 = (size_t)h->n * h->n * h->n;
  // u64 <- u0 (the initial guess), zero64 <- u0 (the right-hand side, restored to zero below)
  PMG_NCUDA(h, cudaMemcpyAsync(h->u64, u0, h->pts() * sizeof(double), kind_in(on_device), h->stream));
  PMG_NCUDA(h, cudaMemcpyAsync(h->zero64, u0, h->pts() * sizeof(double), kind_in(on_device), h->stream));
  PMG_NCUDA(h, cudaMemcpyAsync(h->s.kappa, kappa, sizeof(float) * h->batch, cudaMemcpyHostToDevice, h->stream));
  pmg_options o;
  pfasst_mg_default_options(&o);
  o.smoother = PMG_SMOOTHER_RBGS;
  o.omega = 1.0;
  o.vcycles = 0;  // solved to the tolerance (1e-12)
  o.use_graphs = 0;
  o.autotune = 0;
  const pmg_grid grid{3, h->n, 2};
  const double ih2 = (double)(h->n + 1) * (h->n + 1);
  int rc = PMG_OK;
  for (int b = 0; b < h->batch && rc == PMG_OK; ++b) {
    const double k = kappa[b];
    const double c = k / ((1.0 - 6.0 * k) * ih2);  // kappa = (c/h^2) / (1 + 6 c/h^2)
    rc = pfasst_mg_helmholtz_solve(&grid, c, 1, h->zero64 + b * n3, h->u64 + b * n3, &o, h->stream, nullptr);
    if (rc != PMG_OK) rc = nfail(h, rc, std::string("sub-step solve: ") + pfasst_mg_last_error(nullptr));
  }
  if (rc == PMG_OK) {
    PMG_NCUDA(h, k_net_sub64(h->L(), g, h->u64, h->zero64));  // e0 = u* - u0
    PMG_NCUDA(h, k_net_sample_finish(h->L(), g, h->u64, h->mx, h->xs, h->ts, h->s.kappa));
    const size_t bytes = h->pts() * sizeof(float);
    PMG_NCUDA(h, cudaMemcpyAsync(x, h->xs, bytes, kind_out(on_device), h->stream));
    PMG_NCUDA(h, cudaMemcpyAsync(t, h->ts, bytes, kind_out(on_device), h->stream));
  }
  PMG_NCUDA(h, cudaMemsetAsync(h->zero64, 0, h->pts() * sizeof(double), h->stream));
  PMG_NCUDA(h, cudaStreamSynchronize(h->stream));
  return rc;
}

int pfasst_mg_net_sample(pmg_net_handle h, unsigned long long seed, double kappa_lo, double kappa_hi,
                         int vcycles_max, float *x, float *t, float *kappa, int on_device) {
  if (!h || !x || !t || !kappa) return nfail(h, PMG_ERR_INVALID_ARG, "null handle or array");
  PMG_RET(check_sample_args(h, kappa_lo, kappa_hi, vcycles_max));
  const size_t bytes = h->pts() * sizeof(float);
  PMG_RET(net_draw(h, seed, kappa_lo, kappa_hi, vcycles_max));
  PMG_NCUDA(h, cudaMemcpyAsync(x, h->xs, bytes, kind_out(on_device), h->stream));
  PMG_NCUDA(h, cudaMemcpyAsync(t, h->ts, bytes, kind_out(on_device), h->stream));
  PMG_NCUDA(h, cudaMemcpyAsync(kappa, h->s.kappa, h->batch * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  PMG_NCUDA(h, cudaStreamSynchronize(h->stream));
  return PMG_OK;
}

int pfasst_mg_net_train(pmg_net_handle h, int steps, double lr, unsigned long long seed, double kappa_lo,
                        double kappa_hi, int vcycles_max, int power, int train_bias, double *loss_history) {
  if (!h) return nfail(h, PMG_ERR_INVALID_ARG, "null handle");
  if (power < 0 || power > 3) return nfail(h, PMG_ERR_INVALID_ARG, "power must be 0..3");
  if (steps < 1 || steps > 4096 || !(lr > 0.0))
    return nfail(h, PMG_ERR_INVALID_ARG, "need 1 <= steps <= 4096 and lr > 0");
  PMG_RET(check_sample_args(h, kappa_lo, kappa_hi, vcycles_max));
  PMG_NCUDA(h, cudaMemsetAsync(h->loss, 0, sizeof(double) * steps, h->stream));
  for (int k = 0; k < steps; ++k) {
    PMG_RET(net_draw(h, seed + (unsigned long long)k * 0x9e3779b97f4a7c15ULL, kappa_lo, kappa_hi, vcycles_max));
    PMG_NCUDA(h, cudaMemsetAsync(h->grad, 0, kNetParams * sizeof(float), h->stream));
    PMG_NCUDA(h, k_net_pack(h->L(), h->prm, h->s));
    PMG_NCUDA(h, k_net_grads(h->L(), h->grid(), h->xs, h->ts, h->s.kappa, power, h->prm, h->grad, h->s,
                             h->loss + k));
    PMG_NCUDA(h, k_net_adam(h->L(), h->prm, h->m, h->v, h->grad, ++h->step, (float)lr, 0.9f, 0.999f, 1e-8f,
                            train_bias != 0));
  }
  std::vector<double> hist(steps);
  PMG_NCUDA(h, cudaMemcpyAsync(hist.data(), h->loss, sizeof(double) * steps, cudaMemcpyDeviceToHost, h->stream));
  PMG_NCUDA(h, cudaStreamSynchronize(h->stream));
  for (int k = 0; k < steps; ++k)
    if (!std::isfinite(hist[k])) return nfail(h, PMG_ERR_DIVERGED, "non-finite training loss");
  if (loss_history) std::memcpy(loss_history, hist.data(), sizeof(double) * steps);
  return PMG_OK;
}

int pfasst_mg_net_step(pmg_net_handle h, const float *x, const float *t, const float *kappa, int power, double lr,
                       int train_bias, int on_device, double *loss) {
  if (!h || !x || !t || !kappa) return nfail(h, PMG_ERR_INVALID_ARG, "null handle or array");
  if (power < 0 || power > 3 || !(lr > 0.0)) return nfail(h, PMG_ERR_INVALID_ARG, "need power 0..3 and lr > 0");
  for (int b = 0; b < h->batch; ++b)
    if (!(kappa[b] >= 0.f && kappa[b] <= 1.f / 6.f + 1e-7f))
      return nfail(h, PMG_ERR_INVALID_ARG, "kappa must lie in [0, 1/6]");
  const size_t bytes = h->pts() * sizeof(float);
  PMG_NCUDA(h, cudaMemcpyAsync(h->xs, x, bytes, kind_in(on_device), h->stream));
  PMG_NCUDA(h, cudaMemcpyAsync(h->ts, t, bytes, kind_in(on_device), h->stream));
  PMG_NCUDA(h, cudaMemcpyAsync(h->s.kappa, kappa, h->batch * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  PMG_NCUDA(h, cudaMemsetAsync(h->grad, 0, kNetParams * sizeof(float), h->stream));
  PMG_NCUDA(h, cudaMemsetAsync(h->loss, 0, sizeof(double), h->stream));
  PMG_NCUDA(h, k_net_pack(h->L(), h->prm, h->s));
  PMG_NCUDA(h, k_net_grads(h->L(), h->grid(), h->xs, h->ts, h->s.kappa, power, h->prm, h->grad, h->s, h->loss));
  PMG_NCUDA(h, k_net_adam(h->L(), h->prm, h->m, h->v, h->grad, ++h->step, (float)lr, 0.9f, 0.999f, 1e-8f,
                          train_bias != 0));
  double l = 0.0;
  PMG_NCUDA(h, cudaMemcpyAsync(&l, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  PMG_NCUDA(h, cudaStreamSynchronize(h->stream));
  if (!std::isfinite(l)) return nfail(h, PMG_ERR_DIVERGED, "non-finite training loss");
  if (loss) *loss = l;
  return PMG_OK;
}

long long pfasst_mg_net_launch_count(pmg_net_handle h) { return h ? h->launches : 0; }

int pfasst_mg_net_profile(pmg_net_handle h, int enable, long long min_points) {
  if (!h || min_points < 0) return nfail(h, PMG_ERR_INVALID_ARG, "bad argument");
  h->prof.on = enable != 0;
  h->prof.min_points = min_points;
  return PMG_OK;
}

int pfasst_mg_net_profile_read(pmg_net_handle h, pmg_kernel_stat *out, int capacity, int *count) {
  if (!h || !count || capacity < 0 || (capacity > 0 && !out)) return nfail(h, PMG_ERR_INVALID_ARG, "bad argument");
  PMG_NCUDA(h, cudaStreamSynchronize(h->stream));
  PMG_NCUDA(h, prof_aggregate(h->prof, out, capacity, count));
  return PMG_OK;
}

int pfasst_mg_net_destroy(pmg_net_handle h) {
  if (!h) return PMG_OK;
  if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
  if (h->mem) cudaFree(h->mem);
  delete h;
  return PMG_OK;
}

const char *pfasst_mg_net_last_error(pmg_net_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

int pfasst_mg_set_smoother_net(pmg_handle h, const float *params, int min_n, int calibrate, double *rho_plain,
                               double *rho_net, int *level_mask) {
  if (!h) return fail(nullptr, PMG_ERR_INVALID_ARG, "null handle");
  if (is_batch(h)) return fail(h, PMG_ERR_UNSUPPORTED, "the learned correction is not available on batch handles");
  PMG_CUDA(h, cudaStreamSynchronize(h->stream));
  drop_graph(h->g_pred);
  drop_graph(h->g_pred_spread);
  drop_graph(h->g_iter);
  drop_graph(h->g_loop);
  if (h->net) {
    if (h->net->mem) cudaFree(h->net->mem);
    delete h->net;
    h->net = nullptr;
  }
  if (level_mask) *level_mask = 0;
  if (!params) return PMG_OK;  // plain smoothing everywhere
  if (h->dim != 3 || h->opt.smoother != PMG_SMOOTHER_RBGS || h->opt.nu1 < 2)
    return fail(h, PMG_ERR_UNSUPPORTED, "the learned correction needs dim 3, red-black Gauss-Seidel and nu1 >= 2");
  Hier &H = h->H;
  const int nmin = min_n > 7 ? min_n : 7;
  int lfin = -1, lend = 0;  // eligible levels [lfin, lend): n >= nmin, not the coarsest, 2nd order
  for (int l = 0; l < H.L - 1; ++l)
    if (H.lev[l].n >= nmin && H.lev[l].order != 4) {
      if (lfin < 0) lfin = l;
      lend = l + 1;
    }
  if (lfin < 0) return fail(h, PMG_ERR_INVALID_ARG, "no multigrid level with n >= min_n below the coarsest");
  NetDeploy *d = new (std::nothrow) NetDeploy();
  if (!d) return fail(h, PMG_ERR_OOM, "host allocation failed");
  const size_t per = net_infer_bytes(1, H.lev[lfin]), budget = size_t(1) << 30;
  d->chunk = (int)(budget / per);
  if (d->chunk < 1) d->chunk = 1;
  if (d->chunk > H.batch) d->chunk = H.batch;
  const size_t P = align256(kNetParams * sizeof(float)), bytes = P + net_infer_bytes(d->chunk, H.lev[lfin]);
  if (cudaMalloc(&d->mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete d;
    return fail(h, PMG_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  d->prm = (float *)d->mem;
  d->s = net_infer_carve((char *)d->mem + P, d->chunk, H.lev[lfin]);
  h->net = d;
  PMG_CUDA(h, cudaMemcpyAsync(d->prm, params, kNetParams * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  PMG_CUDA(h, k_net_pack(h->L(), d->prm, d->s));
  double rp = 0.0, rb = 0.0;
  if (calibrate == 2) {
    // judge by the handle's own PFASST iteration: the fine collocation residual after
    // three iterations from the spread initial value, plain and with each level added
    auto run3 = [&](double *res) -> int {
      drop_graph(h->g_pred);
      drop_graph(h->g_pred_spread);
      drop_graph(h->g_iter);
      drop_graph(h->g_loop);
      PMG_RET(spread(h));
      int it = 0;
      const int rc = pfasst_mg_iterate(h, 3, 0.0, &it, res);
      if (rc != PMG_OK && rc != PMG_NOT_CONVERGED) return rc;
      if (!std::isfinite(*res)) *res = INFINITY;
      return PMG_OK;
    };
    PMG_RET(run3(&rp));
    rb = rp;
    for (int l = lfin; l < lend; ++l) {
      d->on[l] = true;
      double r = 0.0;
      PMG_RET(run3(&r));
      if (r < rb) rb = r;
      else d->on[l] = false;
    }
    drop_graph(h->g_pred);
    drop_graph(h->g_pred_spread);
    drop_graph(h->g_iter);
    drop_graph(h->g_loop);
    PMG_RET(spread(h));  // the caller's next iterate starts from the initial value again
  } else {
    PMG_RET(net_measure(h, &rp));
  }
  if (calibrate == 2) {
    // levels chosen above
  } else if (calibrate) {
    rb = rp;
    for (int l = lfin; l < lend; ++l) {  // finest first; keep a level only if it helps
      d->on[l] = true;
      double r = 0.0;
      PMG_RET(net_measure(h, &r));
      if (r < rb) rb = r;
      else d->on[l] = false;
    }
  } else {
    for (int l = lfin; l < lend; ++l) d->on[l] = true;
    PMG_RET(net_measure(h, &rb));
  }
  int mask = 0;
  for (int l = 0; l < H.L - 1; ++l) mask |= d->on[l] ? 1 << l : 0;
  if (rho_plain) *rho_plain = rp;
  if (rho_net) *rho_net = rb;
  if (level_mask) *level_mask = mask;
  if (mask == 0) {  // no level kept: run exactly as without a network
    cudaFree(d->mem);
    delete d;
    h->net = nullptr;
  }
  if (calibrate == 2) {  // graphs captured during the calibration hold earlier level choices
    drop_graph(h->g_pred);
    drop_graph(h->g_pred_spread);
    drop_graph(h->g_iter);
    drop_graph(h->g_loop);
  }
  return PMG_OK;
}

}  // extern "C"

// ----------------------------------------------------------------- allocation-free multigrid solve
//
// Some callers cannot allocate device memory: applications that reserve all of the
// GPU's memory for their own pool allocator at start-up (a raw cudaMalloc then fails or
// fragments their pool), real-time loops in which cudaMalloc / cudaFree would
// synchronise the device and stall every other stream, and deployments whose rules
// forbid allocation after initialisation.  pfasst_mg_helmholtz_solve_noalloc serves
// them: it runs the same V-cycles as pfasst_mg_helmholtz_solve but takes its scratch
// from one fixed device array that is part of this library, so it calls no device
// allocator.

namespace {

// Fixed scratch of the allocation-free solve.  Every GPU that loads this library holds
// these 32 MiB until the process exits.  In host code the name below is only a
// stand-in; its device address comes from cudaGetSymbolAddress.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_base[kNoAllocMaxDevices] = {};

// device address of the scratch on the current device, looked up once per device
int noalloc_base(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, PMG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(nullptr, PMG_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_base[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(nullptr, PMG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_base[dev] = p;
  }
  *out = g_noalloc_base[dev];
  return PMG_OK;
}

// exact inverse of (I - c Lap_h) on the 3^dim grid into a caller array (no heap use);
// same sine eigen-decomposition as coarsest_inverse
void coarsest_inverse_into(int dim, double c, double *out) {
  const int N3 = dim == 1 ? 3 : (dim == 2 ? 9 : 27);
  const long double pi = 3.14159265358979323846264338327950288L;
  long double v[3][3], mu[3];
  for (int k = 0; k < 3; ++k) {
    mu[k] = (2.0L * cosl((k + 1) * pi / 4.0L) - 2.0L) * 16.0L;
    for (int i = 0; i < 3; ++i) v[k][i] = sqrtl(0.5L) * sinl((k + 1) * pi * (i + 1) / 4.0L);
  }
  for (int p = 0; p < N3; ++p)
    for (int q = 0; q < N3; ++q) {
      const int pi3[3] = {p % 3, (p / 3) % 3, p / 9}, qi3[3] = {q % 3, (q / 3) % 3, q / 9};
      long double acc = 0.0L;
      for (int kk = 0; kk < N3; ++kk) {
        const int ks[3] = {kk % 3, (kk / 3) % 3, kk / 9};
        long double lam = 1.0L, prod = 1.0L;
        for (int a = 0; a < dim; ++a) {
          lam -= (long double)c * mu[ks[a]];
          prod *= v[ks[a]][pi3[a]] * v[ks[a]][qi3[a]];
        }
        acc += prod / lam;
      }
      out[p * N3 + q] = (double)acc;
    }
}

// the coarsest-grid inverse travels by value in the kernel's parameters (5832 bytes for
// 27 x 27 FP64 values), so no host buffer has to outlive the call
struct MinvPayload {
  double v[27 * 27];
};

__global__ void store_minv_kernel(MinvPayload p, int count, int f32, void *dst) {
  for (int q = threadIdx.x; q < count; q += blockDim.x) {
    if (f32) ((float *)dst)[q] = (float)p.v[q];
    else ((double *)dst)[q] = p.v[q];
  }
}

}  // namespace

extern "C" int pfasst_mg_helmholtz_solve_noalloc(const pmg_grid *grid, double c, int batch, const double *b,
                                                 double *u, const pmg_options *opt, void *stream, int *cycles_done) {
  pmg_nodes_desc fn{3, 0};
  pmg_levels lv{1, {0, 0}};
  std::string why;
  int rc = validate(grid, &fn, &lv, batch < 1 ? 1 : batch, opt, why);
  if (rc != PMG_OK) return fail(nullptr, rc, why);
  if (batch < 1 || !b || !u || !(c >= 0) || !std::isfinite(c)) return fail(nullptr, PMG_ERR_INVALID_ARG, "bad argument");
  pmg_options o;
  if (opt) o = *opt; else pfasst_mg_default_options(&o);
  if (o.vcycles < 1)
    return fail(nullptr, PMG_ERR_UNSUPPORTED, "the allocation-free solve runs a fixed number of V-cycles (vcycles >= 1)");
  cudaStream_t st = (cudaStream_t)stream;
  Grid g = make_grid(grid->dim, grid->n, grid_order(grid));
  Hier H;
  Plan pl;
  double *bp = nullptr, *up = nullptr;
  void *minv = nullptr;
  pl.add((void **)&bp, (size_t)g.slab * batch * 8);
  pl.add((void **)&up, (size_t)g.slab * batch * 8);
  plan_hier(pl, H, grid->dim, grid->n, batch, o.precision == PMG_PREC_MIXED ? F32 : F64, o.smoother, 0,
            grid_order(grid));
  const int n3 = grid->dim == 1 ? 3 : (grid->dim == 2 ? 9 : 27);
  pl.add(&minv, (size_t)n3 * n3 * H.tsize);
  if (pl.total > kNoAllocScratchBytes)
    return fail(nullptr, PMG_ERR_INVALID_ARG,
                "problem needs " + std::to_string(pl.total) + " bytes of scratch; the allocation-free solve has " +
                    std::to_string(kNoAllocScratchBytes) + " (32 MiB)");
  void *base = nullptr;
  PMG_RET(noalloc_base(&base));
  pl.carve((char *)base);
  // coarsest-grid inverse, computed on the host and stored on the device by a kernel
  // that receives the values as its launch parameters (no host-to-device copy)
  MinvPayload mp;
  coarsest_inverse_into(grid->dim, c, mp.v);
  long long launches = 0;
  Launch Ln{st, &launches, nullptr};
  const long long dense = (long long)g.nz * g.ny * g.n;
  // the array keeps the previous call's contents: clear it (pad columns must be zero)
  if (cudaMemsetAsync(base, 0, pl.total, st) != cudaSuccess)
    return fail(nullptr, PMG_ERR_CUDA, "set-up of the allocation-free solve failed");
  store_minv_kernel<<<1, 256, 0, st>>>(mp, n3 * n3, H.tsize == 4, minv);
  ++launches;
  if (cudaGetLastError() != cudaSuccess || k_pack(Ln, g, b, dense, bp, g.slab, batch) != cudaSuccess ||
      k_pack(Ln, g, u, dense, up, g.slab, batch) != cudaSuccess)
    return fail(nullptr, PMG_ERR_CUDA, "set-up of the allocation-free solve failed");
  MGCtx Mc{Ln, &H, &o, nullptr, nullptr, nullptr, nullptr, nullptr, st};
  PMG_RET(solve_substep(Mc, 0, batch, c, minv, bp, g.slab, nullptr, 0, up, g.slab, nullptr));
  if (k_unpack(Ln, g, up, g.slab, u, dense, batch) != cudaSuccess)
    return fail(nullptr, PMG_ERR_CUDA, "unpack of the allocation-free solve failed");
  if (cycles_done) *cycles_done = o.vcycles;
  return PMG_OK;
}
