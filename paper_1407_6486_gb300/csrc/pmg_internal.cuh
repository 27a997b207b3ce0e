// pmg_internal.cuh -- internal types and kernel launchers of the pfasst_mg library.
//
// Device layout of a grid function with n interior points per axis (n = 2^p - 1):
// [z][y][x] with x padded to pitch = n + 1 = 2^p elements.  The pad element of each
// row is zero and is never written, so rows start on 2^p-element boundaries (16-byte
// aligned for both FP32 and FP64) and the zero Dirichlet wall needs no storage.
// A batch of grid functions is addressed as ptr + b * stride.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <vector>

namespace pmg {

constexpr int kMaxNodes = 9;     // Gauss-Lobatto nodes per level (M + 1)
constexpr int kMaxLevels = 11;   // n <= 1023 -> 9 multigrid levels

enum Prec { F64 = 0, F32 = 1 };

struct Grid {
  int dim;          // 1, 2, 3
  int n;            // interior points per axis
  int pitch;        // n + 1
  int ny, nz;       // n or 1 for missing axes
  long long slab;   // elements of one grid function (nz * ny * pitch)
  double ih2;       // 1 / h^2 = (n + 1)^2
  int order;        // Laplacian stencil: 2 (3 points per axis) or 4 (5 points per axis)
};

inline Grid make_grid(int dim, int n, int order = 2) {
  Grid g;
  g.dim = dim;
  g.n = n;
  g.order = order;
  g.pitch = n + 1;
  g.ny = dim >= 2 ? n : 1;
  g.nz = dim >= 3 ? n : 1;
  g.slab = (long long)g.nz * g.ny * g.pitch;
  g.ih2 = (double)(n + 1) * (double)(n + 1);
  return g;
}

#ifdef __CUDACC__
// binary64 -> binary32 with round-to-nearest-even, done with integer operations on the
// IEEE-754 encodings (sign, biased exponent, significand): GB300 runs the hardware
// conversion on its narrow FP64 pipe, where it bounds the bandwidth of kernels that
// narrow every point.  Bitwise equal to the hardware conversion for every input class
// (normal, subnormal result, overflow to Inf, zero, Inf, NaN stays NaN).
__device__ __forceinline__ float narrow_rn(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffu);
  const unsigned long long m = b & 0xfffffffffffffULL;
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m ? (0x400000u | (unsigned)(m >> 29)) : 0u));
  const int E = e - 1023;
  if (E >= -126) {  // normal result: keep 23 significand bits, round on the 29 dropped ones
    if (E > 127) return __uint_as_float(sign | 0x7f800000u);
    unsigned r = ((unsigned)(E + 127) << 23) | (unsigned)(m >> 29);
    const unsigned rest = (unsigned)(m & 0x1fffffffULL);
    if (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) ++r;  // a carry may reach Inf: correct
    return __uint_as_float(sign | r);
  }
  if (E < -151) return __uint_as_float(sign);  // below half the smallest subnormal
  // subnormal result: (2^52 + m) 2^(E-52) in units of 2^-149
  const unsigned long long full = m | 0x10000000000000ULL;
  const int sh = -97 - E;
  const unsigned long long rem = full & ((1ULL << sh) - 1), half = 1ULL << (sh - 1);
  unsigned r = (unsigned)(full >> sh);
  if (rem > half || (rem == half && (r & 1u))) ++r;
  return __uint_as_float(sign | r);
}

// binary32 -> binary64 on the integer pipe: the widening is exact, so its result is
// fixed by the encodings alone (sign kept; exponent rebiased by 1023 - 127 = 896;
// significand shifted left by 52 - 23 = 29; a subnormal input is normalised by its
// leading one; Inf stays Inf, NaN stays NaN with the quiet bit set).  GB300 runs the
// hardware conversion on its narrow FP64 pipe, next to the FP64 add it feeds.
__device__ __forceinline__ double widen_exact(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
  const unsigned e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  unsigned long long r;
  if (e - 1u < 254u) {  // normal
    r = sign | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  } else if (e == 0xffu) {
    r = sign | 0x7ff0000000000000ULL | (m ? (0x0008000000000000ULL | ((unsigned long long)m << 29)) : 0ULL);
  } else if (m == 0u) {
    r = sign;
  } else {  // subnormal m 2^-149 = 2^(p-149) (1 + fraction), p = position of the leading one
    const int p = 31 - __clz((int)m);
    r = sign | ((unsigned long long)(p + 874) << 52) | (((unsigned long long)m << (52 - p)) & 0xfffffffffffffULL);
  }
  return __longlong_as_double((long long)r);
}

// a multigrid value of storage type T as FP64 (FP32 through widen_exact)
template <typename T>
__device__ __forceinline__ double to_f64(T v) {
  if constexpr (sizeof(T) == 4) return widen_exact(v);
  else return v;
}

template <typename T>
__device__ __forceinline__ T to_storage(double v) {
  if constexpr (sizeof(T) == 4) return narrow_rn(v);
  else return v;
}
#endif

// kernel identifiers for launch accounting and the event profiler
enum KernelId {
  K_RESIDUAL0 = 0, K_JACOBI, K_RBGS, K_RESRESTRICT, K_PROLONG, K_COARSE, K_UPDATE, K_ZERO,
  K_APPLY_A, K_SF_RHS, K_FAS, K_INTERP, K_COLLOC, K_COPY, K_PACK, K_UNPACK, K_INTERP_T,
  K_RBGS3D, K_RESRESTRICT3D, K_PROLONG3D, K_RESID_PT, K_FINE_RHS, K_RBGS3D_ZERO, K_RBGS3D_UPD,
  K_NET_RESID, K_NET_L1, K_NET_L2, K_NET_L3, K_NET_LOSS, K_NET_L3BWD, K_NET_L2BWD, K_NET_WGRAD, K_NET_ADAM,
  K_NET_SAMPLE, K_VTAIL, K_VCOOP, K_COUNT
};

// CUDA-event timing of individual launches on the launching stream (only launches
// that cover at least min_points grid points are recorded).  Eager launches get an
// event pair from a recycled pool; launches recorded while a stream is captured into
// a graph get persistent events recorded by event nodes of the graph, harvested after
// every replay.
struct ProfRec {
  int kid, n, prec;
  long long pts;
  cudaEvent_t a, b;
};
struct ProfDone {
  int kid, n, prec;
  long long pts;
  double ms;
};
struct Profiler {
  bool on = false;
  long long min_points = 0;
  std::vector<cudaEvent_t> pool, persist;
  size_t used = 0;
  std::vector<ProfRec> recs;              // pending eager records
  std::vector<ProfRec> *capture = nullptr;  // set while capturing a graph
  std::vector<ProfDone> done;
  cudaEvent_t take() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  cudaEvent_t take_persistent() {
    cudaEvent_t e;
    cudaEventCreate(&e);
    persist.push_back(e);
    return e;
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
    for (auto e : persist) cudaEventDestroy(e);
  }
};

struct Launch {
  cudaStream_t stream;
  long long *counter;  // incremented per kernel launch (may be null)
  Profiler *prof;      // may be null
};

// records a start event before a launch and the matching end event after it
struct Scope {
  const Launch &L;
  ProfRec rec;
  bool active = false, graph = false;
  Scope(const Launch &L_, KernelId kid, const Grid &g, int batch, int prec) : L(L_) {
    const long long pts = (long long)g.n * g.ny * g.nz * batch;
    if (L.prof && L.prof->on && pts >= L.prof->min_points) {
      rec.kid = kid;
      rec.n = g.n;
      rec.prec = prec;
      rec.pts = pts;
      graph = L.prof->capture != nullptr;
      if (graph) {
        rec.a = L.prof->take_persistent();
        rec.b = L.prof->take_persistent();
        cudaEventRecordWithFlags(rec.a, L.stream, cudaEventRecordExternal);
      } else {
        rec.a = L.prof->take();
        rec.b = L.prof->take();
        cudaEventRecord(rec.a, L.stream);
      }
      active = true;
    }
  }
  cudaError_t done() {
    if (L.counter) ++*L.counter;
    cudaError_t e = cudaGetLastError();
    if (active) {
      if (graph) {
        cudaEventRecordWithFlags(rec.b, L.stream, cudaEventRecordExternal);
        L.prof->capture->push_back(rec);
      } else {
        cudaEventRecord(rec.b, L.stream);
        L.prof->recs.push_back(rec);
      }
    }
    return e;
  }
};

// sub-step right-hand side coefficients:
//   q_m = sum_j W[m][j] F_j (+ tau_{m+1} - tau_m) (- U_{m+1} when sub_next)
// Full solves: W = dt (Q[m+1][j] - Q[m][j]) - [j == m+1] dt_m and sub_next = 0, so that
// u_m + q_m is the right-hand side of the sub-step equation.  Fixed V-cycle counts:
// W = dt (Q[m+1][j] - Q[m][j]) and sub_next = 1, so that u_m + q_m is directly the
// initial residual b - (I - dt_m A) u^k_{m+1} (using F_{m+1} = A u^k_{m+1}).
struct SFCoef {
  int s;                                 // nodes
  int sub_next;
  double W[kMaxNodes - 1][kMaxNodes];
};

// collocation residual coefficients: r_m = U_0 + sum_i dtQ[m][i] F_i - U_m
struct ResCoef {
  int s;
  double dtQ[kMaxNodes][kMaxNodes];
  double dS[kMaxNodes - 1][kMaxNodes];  // dt (Q[m+1][j] - Q[m][j]): node-to-node quadrature S
};

// FAS restriction coefficients (coarse node j <-> fine node map[j])
struct FASCoef {
  int sf, sc;
  int map[kMaxNodes];
  double dtQf[kMaxNodes][kMaxNodes];     // rows map[j] of dt * Q_fine
  double dtQc[kMaxNodes][kMaxNodes];     // dt * Q_coarse
  double nu;
  int zero_rows;                         // bit j: rows j of dtQf and dtQc are zero, so tau_j = 0
};

// coarse-correction interpolation: U_f,m += sum_j T[m][j] I_x (U_c,j - U_c0,j)
struct InterpCoef {
  int sf, sc, order;
  double T[kMaxNodes][kMaxNodes];
  float T32[kMaxNodes][kMaxNodes];  // the same weights rounded to FP32
};

// ---- multigrid kernels (precision of e, f chosen by Prec) ----
cudaError_t k_residual0(const Launch &L, const Grid &g, double c, Prec pr, const double *um, long long sum,
                        const double *qm, long long sq, const double *u1, long long s1, void *f, int batch,
                        unsigned long long *rnorm, unsigned long long *bnorm);
// threads: block size of the one-point-per-thread smoothers (128, 256, 512, ...)
cudaError_t k_smooth_jacobi(const Launch &L, const Grid &g, double c, double omega, Prec pr, const void *ein,
                            void *eout, const void *f, int batch, bool first, int threads = 256);
cudaError_t k_smooth_rbgs(const Launch &L, const Grid &g, double c, double omega, Prec pr, void *e, const void *f,
                          int batch, int colour, bool first, int threads = 256);
cudaError_t k_residual_restrict(const Launch &L, const Grid &gf, const Grid &gc, double c, Prec pr, const void *e,
                                const void *f, void *fc, int batch);
cudaError_t k_prolong_add(const Launch &L, const Grid &gf, const Grid &gc, Prec pr, const void *ec, void *e, int batch);
cudaError_t k_coarse_solve(const Launch &L, const Grid &g3, Prec pr, const void *minv, const void *f, void *e,
                           int batch);
cudaError_t k_update_u(const Launch &L, const Grid &g, Prec pr, double *u, long long su, const void *e, int batch,
                       const int *active);
cudaError_t k_zero(const Launch &L, const Grid &g, Prec pr, void *e, int batch);

// tiled 3D kernels for large batched grids (stencil3d.cu)
constexpr int kTiled3dMinN = 63;
// zchunk: z planes per CTA of the fused sweep (0 = default); threads: 256 or 512
// threads per CTA for the full-row variant
cudaError_t k_rbgs_sweep3d(const Launch &L, const Grid &g, double c, double omega, Prec pr, const void *ein,
                           void *eout, const void *f, double *u, long long su, int batch, bool zero, bool update_u,
                           int zchunk = 0, int threads = 256);
bool rbgs_rows_supported(const Grid &g);
// the same fused sweep with TMA-staged planes (sweep_tma.cu): FP32, pitch 128 or 256
bool rbgs_tma_supported(const Grid &g, Prec pr);
// threads per CTA: two x points per thread, or four (quad)
int rbgs_tma_threads(const Grid &g, bool quad);
cudaError_t k_rbgs_sweep3d_tma(const Launch &L, const Grid &g, double c, double omega, const void *ein, void *eout,
                               const void *f, double *u, long long su, int batch, bool zero, bool update_u,
                               int zchunk, bool quad);
// nonzero if a bounded device-side wait of a sweep timed out since the last call (clears it)
int sweep_timeouts();
// the same for the TMA-staged interpolation of the coarse correction
int interp_timeouts();
cudaError_t k_resrestrict3d(const Launch &L, const Grid &gf, const Grid &gc, double c, Prec pr, const void *e,
                            const void *f, void *fc, int batch);
// the same residual + full weighting with TMA-staged planes (sweep_tma.cu): FP32, pitch >= 128
bool resrestrict_tma_supported(const Grid &gf, Prec pr);
cudaError_t k_resrestrict3d_tma(const Launch &L, const Grid &gf, const Grid &gc, double c, const void *e, const void *f,
                                void *fc, int batch);
cudaError_t k_prolong3d(const Launch &L, const Grid &gf, const Grid &gc, Prec pr, const void *ec, void *e, int batch);

// ---- SDC / PFASST kernels (FP64) ----
cudaError_t k_apply_A(const Launch &L, const Grid &g, double nu, const double *u, long long su, double *F,
                      long long sF, int batch);
cudaError_t k_sf_rhs(const Launch &L, const Grid &g, const SFCoef &cf, const double *F, const double *U, long long sF,
                     const double *tau, long long stau, double *q, long long sq, int batch);
// pointwise initial residual f = (T)(u_m + q_m) of the sub-step equation
cudaError_t k_resid_pt(const Launch &L, const Grid &g, Prec pr, const double *um, long long sum, const double *qm,
                       long long sq, void *f, int batch);
// FAS restriction with a stored fine F; tauf (stride sfine, may be null) is the fine
// level's own FAS correction, added to its integral when the fine level is itself a
// coarse level of a deeper hierarchy
cudaError_t k_fas_restrict(const Launch &L, const Grid &gf, const Grid &gc, const FASCoef &cf, const double *Uf,
                           const double *Ff, long long sfine, double *Uc, double *Fc, double *tau, double *Uc0,
                           long long scoarse, int batch, const double *tauf = nullptr);
// coarse-correction interpolation in two steps: in time on the coarse grid (dU in the
// precision pr), then in space onto every fine node m >= m0, added to U_f (m0 = 1 when
// the fine node 0 is overwritten by the send-forward right after)
cudaError_t k_interp_time(const Launch &L, const Grid &gc, const InterpCoef &cf, Prec pr, const double *Uc,
                          const double *Uc0, long long scoarse, void *dU, int batch, int m0 = 0);
cudaError_t k_interp_space_add(const Launch &L, const Grid &gf, const Grid &gc, int order, int sf, Prec pr,
                               const void *dU, double *Uf, long long sfine, int batch, int m0 = 0);
// fine level without stored F (fixed V-cycle counts): residual + next right-hand sides
// chained: U[b][0] is a copy of U[b-1][S-1] for b >= 1 (after the send-forward); node 0's
// Laplacian is then taken over from the previous slice (same results)
cudaError_t k_fine_rhs_residual(const Launch &L, const Grid &g, const ResCoef &cf, double nu, const double *U,
                                long long stride, double *q, long long sq, int batch, unsigned long long *res,
                                bool chained = false);
cudaError_t k_fas_restrict_u(const Launch &L, const Grid &gf, const Grid &gc, const FASCoef &cf, const double *Uf,
                             long long sfine, double *Uc, double *Fc, double *tau, double *Uc0, long long scoarse,
                             int batch);
cudaError_t k_colloc_residual(const Launch &L, const Grid &g, const ResCoef &cf, const double *U, const double *F,
                              long long stride, int batch, unsigned long long *out);
// compares narrow_rn with the hardware FP64 -> FP32 conversion on `count` generated
// inputs; adds the number of differing results to *bad (device memory)
cudaError_t k_narrow_check(cudaStream_t st, long long count, unsigned long long seed, unsigned long long *bad);
// compares widen_exact with the hardware FP32 -> FP64 conversion on every one of the 2^32
// float bit patterns (NaN inputs: both results must be NaN); adds the mismatches to *bad
cudaError_t k_widen_check(cudaStream_t st, unsigned long long *bad);
cudaError_t k_copy(const Launch &L, const Grid &g, const double *src, long long ss, double *dst, long long sd,
                   int batch);
cudaError_t k_pack(const Launch &L, const Grid &g, const double *dense, long long sdense, double *pad, long long spad,
                   int batch);
cudaError_t k_unpack(const Launch &L, const Grid &g, const double *pad, long long spad, double *dense,
                     long long sdense, int batch);


// ---- all V-cycles of a single-grid sub-step solve in one persistent launch (vcycle_coop.cu) ----
// red-black Gauss-Seidel (nu1 >= 1), 2D or 3D, second order
bool vcycle_coop_supported(const Grid &g0, int levels, int smoother_rbgs, int nu1);
// nv V(nu1, nu2)-cycles for (I - c Lap) e = f[0] on levels lev[0..nlev-1] (one grid each,
// e[l], f[l] and the residual scratch r[l] in the precision pr; e[0] from zero), then
// u += e[0] if u is not null;
// count: a device word for the grid barrier (zeroed here, on the stream)
cudaError_t k_vcycle_coop(const Launch &L, const Grid *lev, int nlev, Prec pr, double c, double omega, int nu1,
                          int nu2, int nv, void *const *e, void *const *f, void *const *r, const void *minv,
                          double *u, unsigned *count);
// nonzero if a grid barrier of the persistent V-cycle timed out since the last call (clears it)
int coop_timeouts();

// ---- bottom of a V-cycle in one launch (tail.cu) ----
// levels top .. 3^d of one grid per CTA in shared memory: offsets (elements) of the
// dense e, e2 (Jacobi), f and residual arrays of every tail level
constexpr size_t kVTailMaxSmem = 200 * 1024;
struct VTailDesc {
  int nlev = 0;
  int n[kMaxLevels] = {};
  int off_e[kMaxLevels] = {}, off_e2[kMaxLevels] = {}, off_f[kMaxLevels] = {}, off_r[kMaxLevels] = {};
  size_t smem_elems = 0;
  double c = 0, omega = 1;
  int smoother = 1, nu1 = 2, nu2 = 1;  // smoother 0 = weighted Jacobi, 1 = red-black Gauss-Seidel
};
// fills d for nlev levels from n_top; returns the shared-memory bytes
size_t vtail_plan(int dim, int n_top, int nlev, int smoother, size_t tsize, VTailDesc &d);
// e (top level, padded layout) = V-cycle correction for right-hand side f, starting
// from e_in (may equal e) or from zero (e_in null)
cudaError_t k_vcycle_tail(const Launch &L, const Grid &g_top, const VTailDesc &d, Prec pr, const void *minv,
                          const void *f, const void *e_in, void *e, int batch);

// ---- learned correction network (learned.cu) ----
// Flat FP32 parameter vector: W1[16][27], b1[16], W2[16][27][16] ([out][tap][in]),
// b2[16], W3[27][16] ([tap][in]), b3; tap = (dz+1)*9 + (dy+1)*3 + (dx+1).
constexpr int kNetC = 16;
constexpr int kNetW1 = 0, kNetB1 = kNetW1 + kNetC * 27, kNetW2 = kNetB1 + kNetC,
              kNetB2 = kNetW2 + kNetC * 27 * kNetC, kNetW3 = kNetB2 + kNetC, kNetB3 = kNetW3 + 27 * kNetC,
              kNetParams = kNetB3 + 1;

// batch of n^3 grids; the network input and output grid functions are addressed as
// b * slab + (z * n + y) * pitch + x (dense: pitch = n, slab = n^3; the padded level
// layout: pitch = n + 1); hidden activations are dense [b][z][y][x][16] BF16.
struct NetGrid {
  int batch, n, pitch;
  long long slab;
};

struct NetScratch {
  __nv_bfloat16 *a1 = nullptr, *a2 = nullptr, *gz2b = nullptr, *w2f = nullptr, *w2t = nullptr;
  float *gz2 = nullptr, *gz1 = nullptr, *y = nullptr, *w = nullptr, *gy = nullptr, *x = nullptr, *tmp = nullptr;
  float *kappa = nullptr;
};

// scratch of the training kernels (batch dense n^3 grids) / of the correction step
size_t net_train_bytes(int batch, int n);
NetScratch net_train_carve(void *base, int batch, int n);
size_t net_infer_bytes(int batch, const Grid &g);
NetScratch net_infer_carve(void *base, int batch, const Grid &g);

void net_init_params(float *prm, unsigned long long seed);  // host, He-scaled normals, zero biases
cudaError_t k_net_pack(const Launch &L, const float *prm, const NetScratch &s);
cudaError_t k_net_forward(const Launch &L, const NetGrid &g, const float *x, const float *prm, const NetScratch &s,
                          float *y);
// loss 0.5 mean((Ahat_kappa_b^power (y - t))^2) and its gradient, added to grad / *loss
cudaError_t k_net_grads(const Launch &L, const NetGrid &g, const float *x, const float *t, const float *kappa,
                        int power, const float *prm, float *grad, const NetScratch &s, double *loss);
cudaError_t k_net_adam(const Launch &L, float *prm, float *m, float *v, const float *grad, int step, float lr,
                       float b1, float b2, float eps, bool train_bias);
// synthetic training pairs: kappa_b uniform in [lo, hi]; t = one red-black Gauss-Seidel
// sweep of Ahat t = 0 applied to uniform noise; x = Ahat t
cudaError_t k_net_sample(const Launch &L, const NetGrid &g, unsigned long long seed, float klo, float khi, float *x,
                         float *t, float *kappa);
// the kappa of grid b of a sample (as the sample kernels draw it), and its V-cycle count
float net_sample_kappa(unsigned long long seed, float klo, float khi, int b);
int net_sample_vcycles(unsigned long long seed, int vmax, int b);
// multigrid-shaped training pairs, in three steps: FP64 noise u (dense); the caller runs
// V-cycles of (I - c Lap) u = 0 on u; then t = u / max|u| per grid, one red-black sweep
// of Ahat t = 0, x = Ahat t (mx: batch scratch words)
cudaError_t k_net_sample_noise64(const Launch &L, const NetGrid &g, unsigned long long seed, double *u);
cudaError_t k_net_sample_finish(const Launch &L, const NetGrid &g, const double *u, unsigned long long *mx,
                                float *x, float *t, const float *kappa);
// a -= b on the dense FP64 grids of a net batch
cudaError_t k_net_sub64(const Launch &L, const NetGrid &g, double *a, const double *b);
// correction step on a multigrid level: x = D^-1 (f - (I - c Lap) e), e += net(x)
cudaError_t k_net_correct(const Launch &L, const Grid &g, double c, Prec pr, void *e, const void *f, int batch,
                          const float *prm, const NetScratch &s);
// calibration helpers on a level: e = uniform noise in [-1, 1] (walls zero); max |e|
cudaError_t k_net_noise(const Launch &L, const Grid &g, Prec pr, void *e, int batch, unsigned long long seed);
cudaError_t k_net_maxabs(const Launch &L, const Grid &g, Prec pr, const void *e, int batch, unsigned long long *out);

}  // namespace pmg
