// kernels.cu -- CUDA kernels of the pfasst_mg library (sm_103a).
//
// Generic, batched stencil kernels for every level of the space-time hierarchy:
// the sub-step residual of Eq. SDCcompactLIII, weighted-Jacobi and red-black
// Gauss-Seidel smoothing, residual + full-weighting restriction, d-linear
// prolongation, the exact 3^d coarsest-grid solve (multigrid of Sec. 4.1.1), the
// F = nu Lap_h U evaluation, the node-to-node quadrature S F of Eq. sdc-be, the FAS
// restriction (Sec. 2.3), the 4th-order space / Lagrange time interpolation of the
// coarse correction (Sec. 4.2.1) and the collocation residual of Eq. resid.
//
// Thread mapping: x (unit stride) across threadIdx.x, rows across (blockIdx.y,
// threadIdx.y), (z, batch) across blockIdx.z, with grid-stride loops so any size is
// covered.  All accesses stay inside the interior of each grid; the pad column is
// never written.
#include "pmg_internal.cuh"
#include "tma.cuh"

namespace pmg {
namespace {

__device__ int g_interp_timeout;  // set by a timed-out wait of interp_space3d_tma_kernel

#define PMG_FOR_POINTS(g, batch)                                                                   \
  for (int zb = blockIdx.z; zb < (g).nz * (batch); zb += gridDim.z)                                \
    for (int j = blockIdx.y * blockDim.y + threadIdx.y; j < (g).ny; j += gridDim.y * blockDim.y) \
      for (int i = threadIdx.x; i < (g).n; i += blockDim.x)

#define PMG_POINT(g)                 \
  const int k = zb % (g).nz;         \
  const int b = zb / (g).nz;         \
  const long long off = ((long long)k * (g).ny + j) * (g).pitch + i

void config(const Grid &g, int batch, dim3 &grid, dim3 &block, int threads = 256) {
  // a multiple of 32 threads per block always, so every warp is full (the reductions
  // use full-warp shuffles); small grids simply leave rows idle
  int bx = g.pitch < threads ? g.pitch : threads;
  int by = threads / bx;
  block = dim3(bx, by, 1);
  int gy = (g.ny + by - 1) / by;
  long long gz = (long long)g.nz * batch;
  if (gz > 65535) gz = 65535;
  if (gz < 1) gz = 1;
  grid = dim3(1, gy, (unsigned)gz);
}

// sum of the 2*DIM neighbours, zero outside the interior (Dirichlet 0)
template <int DIM, typename T>
__device__ __forceinline__ T nbsum(const T *__restrict__ u, const Grid &g, int i, int j, int k, long long off) {
  T s = (i > 0 ? u[off - 1] : T(0)) + (i < g.n - 1 ? u[off + 1] : T(0));
  if (DIM >= 2) s += (j > 0 ? u[off - g.pitch] : T(0)) + (j < g.n - 1 ? u[off + g.pitch] : T(0));
  if (DIM >= 3) {
    const long long pl = (long long)g.ny * g.pitch;
    s += (k > 0 ? u[off - pl] : T(0)) + (k < g.n - 1 ? u[off + pl] : T(0));
  }
  return s;
}

// one axis of h^2 times the fourth-order Laplacian at index c of an axis of length len
// (stride st): (-u_{c-2} + 16 u_{c-1} - 30 u_c + 16 u_{c+1} - u_{c+2}) / 12.  The wall
// value is zero; the one point beyond the wall that the stencil reaches is the odd
// reflection -u of its mirror image, which for the first and last point of the axis is
// the point itself (Sec. 4.2 stencil; the reflection keeps sine modes eigenvectors).
template <typename T>
__device__ __forceinline__ T axis4(const T *__restrict__ u, long long off, int c, int len, long long st, T uc) {
  const T m1 = c >= 1 ? u[off - st] : T(0);
  const T m2 = c >= 2 ? u[off - 2 * st] : (c == 0 ? -uc : T(0));
  const T p1 = c + 1 < len ? u[off + st] : T(0);
  const T p2 = c + 2 < len ? u[off + 2 * st] : (c == len - 1 ? -uc : T(0));
  return (-m2 + T(16) * m1 - T(30) * uc + T(16) * p1 - p2) / T(12);
}

// h^2 times the fourth-order Laplacian at one point
template <int DIM, typename T>
__device__ __forceinline__ T lap4_h2(const T *__restrict__ u, const Grid &g, int i, int j, int k, long long off) {
  const T uc = u[off];
  T s = axis4(u, off, i, g.n, 1, uc);
  if (DIM >= 2) s += axis4(u, off, j, g.ny, g.pitch, uc);
  if (DIM >= 3) s += axis4(u, off, k, g.nz, (long long)g.ny * g.pitch, uc);
  return s;
}

// h^2 Lap_h u at one point, for the grid's stencil order
template <int DIM, typename T>
__device__ __forceinline__ T lap_h2(const T *__restrict__ u, const Grid &g, int i, int j, int k, long long off) {
  if (g.order == 4) return lap4_h2<DIM>(u, g, i, j, k, off);
  return nbsum<DIM>(u, g, i, j, k, off) - T(2 * DIM) * u[off];
}

// -h^2 times the diagonal entry of Lap_h: 2 DIM, or for the fourth-order stencil 30/12
// per axis (29/12 where the point is first or last on the axis: its reflected image)
template <int DIM, typename T>
__device__ __forceinline__ T diag_h2(const Grid &g, int i, int j, int k) {
  if (g.order != 4) return T(2 * DIM);
  T d = (i == 0 || i == g.n - 1) ? T(29) / T(12) : T(30) / T(12);
  if (DIM >= 2) d += (j == 0 || j == g.ny - 1) ? T(29) / T(12) : T(30) / T(12);
  if (DIM >= 3) d += (k == 0 || k == g.nz - 1) ? T(29) / T(12) : T(30) / T(12);
  return d;
}

// max-reduce nonnegative doubles (NaN wins) across a warp, one atomic per warp
__device__ __forceinline__ void warp_max_atomic(double v, unsigned long long *dst) {
  const unsigned full = 0xffffffffu;
  for (int o = 16; o > 0; o >>= 1) {
    double w = __shfl_xor_sync(full, v, o);
    if (!(w <= v)) v = w;  // NaN propagates
  }
  if ((threadIdx.x & 31) == 0 && v != 0.0) atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

// ------------------------------------------------------------------ multigrid

// f = (u_m + q_m) - (I - c Lap_h) u_{m+1}  (FP64 arithmetic, stored as TO)
template <int DIM, typename TO>
__global__ void residual0_kernel(Grid g, double c, const double *__restrict__ um, long long sum,
                                 const double *__restrict__ qm, long long sq, const double *__restrict__ u1,
                                 long long s1, TO *__restrict__ f, int batch, unsigned long long *rnorm,
                                 unsigned long long *bnorm) {
  const double a = c * g.ih2;
  for (int zb = blockIdx.z; zb < g.nz * batch; zb += gridDim.z) {
    const int k = zb % g.nz, b = zb / g.nz;
    double rmax = 0.0, bmax = 0.0;
    for (int j = blockIdx.y * blockDim.y + threadIdx.y; j < g.ny; j += gridDim.y * blockDim.y)
      for (int i = threadIdx.x; i < g.n; i += blockDim.x) {
        const long long off = ((long long)k * g.ny + j) * g.pitch + i;
        const double *U1 = u1 + b * s1;
        const double uc = U1[off];
        const double Lu = uc - a * lap_h2<DIM>(U1, g, i, j, k, off);
        const double rhs = um[b * sum + off] + (qm ? qm[b * sq + off] : 0.0);
        const double r = rhs - Lu;
        f[b * g.slab + off] = (TO)r;
        const double ar = fabs(r), ab = fabs(rhs);
        if (!(ar <= rmax)) rmax = ar;
        if (!(ab <= bmax)) bmax = ab;
      }
    if (rnorm) {
      warp_max_atomic(rmax, rnorm + b);
      warp_max_atomic(bmax, bnorm + b);
    }
  }
}

template <int DIM, typename T>
__global__ void jacobi_kernel(Grid g, T c, T omega, const T *__restrict__ ein, T *__restrict__ eout,
                              const T *__restrict__ f, int batch, int first) {
  const T a = c * (T)g.ih2;
  const T D = T(1) + T(2 * DIM) * a;
  const T wD = omega / D;
  PMG_FOR_POINTS(g, batch) {
    PMG_POINT(g);
    const long long o = b * g.slab + off;
    if (g.order == 4) {  // diagonal varies next to the walls
      const T Dp = T(1) + a * diag_h2<DIM, T>(g, i, j, k);
      if (first) {
        eout[o] = omega * f[o] / Dp;
      } else {
        const T *E = ein + b * g.slab;
        const T ec = E[off];
        eout[o] = ec + omega * (f[o] - (ec - a * lap_h2<DIM>(E, g, i, j, k, off))) / Dp;
      }
    } else if (first) {
      eout[o] = wD * f[o];
    } else {
      const T *E = ein + b * g.slab;
      const T ec = E[off];
      const T Le = ec - a * (nbsum<DIM>(E, g, i, j, k, off) - T(2 * DIM) * ec);
      eout[o] = ec + wD * (f[o] - Le);
    }
  }
}

// red = (i+j+k) even in 1-based interior indices of the existing axes.  On a grid with
// the fourth-order stencil the colour is (i+j+k) mod 3 instead (three half-sweeps):
// points of one colour are at least 3 apart on every axis, outside each other's stencil.
template <int DIM, typename T>
__global__ void rbgs_kernel(Grid g, T c, T omega, T *e, const T *__restrict__ f, int batch, int colour,
                            int first) {
  const T a = c * (T)g.ih2;
  const T D = T(1) + T(2 * DIM) * a;
  PMG_FOR_POINTS(g, batch) {
    PMG_POINT(g);
    const long long o = b * g.slab + off;
    const int par = g.order == 4 ? (i + j + k + DIM) % 3 : (i + j + k + DIM) & 1;
    if (par != colour) {
      if (first && colour == 0) e[o] = T(0);
      continue;
    }
    if (g.order == 4) {
      const T Dp = T(1) + a * diag_h2<DIM, T>(g, i, j, k);
      if (first && colour == 0) {
        e[o] = omega * f[o] / Dp;
        continue;
      }
      const T *E = e + b * g.slab;
      const T ec = E[off];
      e[o] = ec + omega * (f[o] - (ec - a * lap_h2<DIM>(E, g, i, j, k, off))) / Dp;
      continue;
    }
    if (first && colour == 0) {
      e[o] = omega * (f[o] / D);
      continue;
    }
    const T *E = e + b * g.slab;
    const T gs = (f[o] + a * nbsum<DIM>(E, g, i, j, k, off)) / D;
    e[o] = (T(1) - omega) * e[o] + omega * gs;
  }
}

// fc(I) = sum of full-weighting taps of r = f - (I - c Lap_h) e around fine 2I+1
template <int DIM, typename T>
__global__ void resrestrict_kernel(Grid gf, Grid gc, T c, const T *__restrict__ e, const T *__restrict__ f,
                                   T *__restrict__ fc, int batch) {
  const T a = c * (T)gf.ih2;
  const T w3[3] = {T(0.25), T(0.5), T(0.25)};
  PMG_FOR_POINTS(gc, batch) {
    PMG_POINT(gc);
    const T *E = e + b * gf.slab;
    const T *Fp = f + b * gf.slab;
    T acc = T(0);
    for (int cz = (DIM >= 3 ? -1 : 0); cz <= (DIM >= 3 ? 1 : 0); ++cz)
      for (int cy = (DIM >= 2 ? -1 : 0); cy <= (DIM >= 2 ? 1 : 0); ++cy)
        for (int cx = -1; cx <= 1; ++cx) {
          const int fi = 2 * i + 1 + cx;
          const int fj = DIM >= 2 ? 2 * j + 1 + cy : 0;
          const int fk = DIM >= 3 ? 2 * k + 1 + cz : 0;
          const long long fo = ((long long)fk * gf.ny + fj) * gf.pitch + fi;
          const T ec = E[fo];
          const T r = Fp[fo] - (ec - a * lap_h2<DIM>(E, gf, fi, fj, fk, fo));
          T w = w3[cx + 1];
          if (DIM >= 2) w *= w3[cy + 1];
          if (DIM >= 3) w *= w3[cz + 1];
          acc += w * r;
        }
    fc[b * gc.slab + off] = acc;
  }
}

// linear interpolation taps of fine 0-based index i onto coarse 0-based indices
__device__ __forceinline__ int lin_taps(int i, int nc, int *idx, float *w) {
  const int i1 = i + 1;
  if ((i1 & 1) == 0) {
    idx[0] = i1 / 2 - 1;
    w[0] = 1.0f;
    return 1;
  }
  int t = 0;
  const int lo = (i1 - 1) / 2 - 1, hi = (i1 + 1) / 2 - 1;
  if (lo >= 0) { idx[t] = lo; w[t] = 0.5f; ++t; }
  if (hi < nc) { idx[t] = hi; w[t] = 0.5f; ++t; }
  return t;
}

template <int DIM, typename T>
__global__ void prolong_kernel(Grid gf, Grid gc, const T *__restrict__ ec, T *__restrict__ e, int batch) {
  PMG_FOR_POINTS(gf, batch) {
    PMG_POINT(gf);
    int ix[2], iy[2] = {0, 0}, iz[2] = {0, 0};
    float wx[2], wy[2] = {1.f, 1.f}, wz[2] = {1.f, 1.f};
    const int tx = lin_taps(i, gc.n, ix, wx);
    const int ty = DIM >= 2 ? lin_taps(j, gc.n, iy, wy) : 1;
    const int tz = DIM >= 3 ? lin_taps(k, gc.n, iz, wz) : 1;
    const T *EC = ec + b * gc.slab;
    T acc = T(0);
    for (int cz = 0; cz < tz; ++cz)
      for (int cy = 0; cy < ty; ++cy)
        for (int cx = 0; cx < tx; ++cx)
          acc += T(wx[cx] * wy[cy] * wz[cz]) * EC[((long long)iz[cz] * gc.ny + iy[cy]) * gc.pitch + ix[cx]];
    e[b * gf.slab + off] += acc;
  }
}

// exact solve on the 3^d grid: e = Minv f (Minv dense, row-major N3 x N3)
template <int DIM, typename T>
__global__ void coarse_solve_kernel(Grid g, const T *__restrict__ minv, const T *__restrict__ f, T *__restrict__ e,
                                    int batch) {
  constexpr int N3 = DIM == 1 ? 3 : (DIM == 2 ? 9 : 27);
  PMG_FOR_POINTS(g, batch) {
    PMG_POINT(g);
    const int p = (k * 3 + j) * 3 + i;
    const T *Fb = f + b * g.slab;
    T acc = T(0);
    for (int q = 0; q < N3; ++q) {
      const int qi = q % 3, qj = (q / 3) % 3, qk = q / 9;
      acc += minv[p * N3 + q] * Fb[((long long)qk * g.ny + qj) * g.pitch + qi];
    }
    e[b * g.slab + off] = acc;
  }
}

template <typename T>
__global__ void resid_pt_kernel(Grid g, const double *__restrict__ um, long long sum, const double *__restrict__ qm,
                                long long sq, T *__restrict__ f, int batch) {
  PMG_FOR_POINTS(g, batch) {
    PMG_POINT(g);
    f[b * g.slab + off] = to_storage<T>(um[b * sum + off] + qm[b * sq + off]);
  }
}

template <typename T>
__global__ void update_u_kernel(Grid g, double *__restrict__ u, long long su, const T *__restrict__ e, int batch,
                                const int *__restrict__ active) {
  PMG_FOR_POINTS(g, batch) {
    PMG_POINT(g);
    if (active && !active[b]) continue;
    if constexpr (sizeof(T) == 4) u[b * su + off] += widen_exact(e[b * g.slab + off]);
    else u[b * su + off] += e[b * g.slab + off];
  }
}

template <typename T>
__global__ void zero_kernel(Grid g, T *__restrict__ e, int batch) {
  PMG_FOR_POINTS(g, batch) {
    PMG_POINT(g);
    e[b * g.slab + off] = T(0);
  }
}

// ------------------------------------------------------------------ SDC / PFASST

template <int DIM>
__global__ void apply_A_kernel(Grid g, double nu, const double *__restrict__ u, long long su, double *__restrict__ F,
                               long long sF, int batch) {
  const double a = nu * g.ih2;
  PMG_FOR_POINTS(g, batch) {
    PMG_POINT(g);
    const double *U = u + b * su;
    F[b * sF + off] = a * lap_h2<DIM>(U, g, i, j, k, off);
  }
}

// S = node count as a template parameter: no predicated-off FP64 work
template <int S>
__global__ void sf_rhs_kernel(Grid g, SFCoef cf, const double *__restrict__ F, const double *__restrict__ U,
                              long long sF, const double *__restrict__ tau, long long stau, double *__restrict__ q,
                              long long sq, int batch) {
  PMG_FOR_POINTS(g, batch) {
    PMG_POINT(g);
    double Fv[S];
#pragma unroll
    for (int jn = 0; jn < S; ++jn) Fv[jn] = F[b * sF + jn * g.slab + off];
    double tprev = tau ? tau[b * stau + off] : 0.0;
#pragma unroll
    for (int m = 0; m < S - 1; ++m) {
      double acc = 0.0;
#pragma unroll
      for (int jn = 0; jn < S; ++jn) acc += cf.W[m][jn] * Fv[jn];
      if (tau) {
        const double tnext = tau[b * stau + (m + 1) * g.slab + off];
        acc += tnext - tprev;
        tprev = tnext;
      }
      if (cf.sub_next) acc -= U[b * sF + (m + 1) * g.slab + off];
      q[b * sq + m * g.slab + off] = acc;
    }
  }
}

// per coarse point: U_c,j = U_f,map j (injection), F_c,j = A_c U_c,j,
// tau_j = inject(tau_f,map j + sum_i dtQf[j][i] F_f,i) - sum_i dtQc[j][i] F_c,i
// (tau_f = 0 on the finest level)
template <int DIM>
__global__ void fas_restrict_kernel(Grid gf, Grid gc, FASCoef cf, const double *__restrict__ Uf,
                                    const double *__restrict__ Ff, long long sfine, double *__restrict__ Uc,
                                    double *__restrict__ Fc, double *__restrict__ tau, double *__restrict__ Uc0,
                                    long long scoarse, int batch, const double *__restrict__ tauf) {
  const double ac = cf.nu * gc.ih2;
  const long long plf = (long long)gf.ny * gf.pitch;
  PMG_FOR_POINTS(gc, batch) {
    PMG_POINT(gc);
    const int fi = 2 * i + 1, fj = DIM >= 2 ? 2 * j + 1 : 0, fk = DIM >= 3 ? 2 * k + 1 : 0;
    const long long fo = ((long long)fk * gf.ny + fj) * gf.pitch + fi;
    double Fcv[kMaxNodes];
    for (int jn = 0; jn < cf.sc; ++jn) {
      const double *U = Uf + b * sfine + cf.map[jn] * gf.slab;
      const double uc = U[fo];
      double s = (i > 0 ? U[fo - 2] : 0.0) + (i < gc.n - 1 ? U[fo + 2] : 0.0);
      if (DIM >= 2) s += (j > 0 ? U[fo - 2 * gf.pitch] : 0.0) + (j < gc.n - 1 ? U[fo + 2 * gf.pitch] : 0.0);
      if (DIM >= 3) s += (k > 0 ? U[fo - 2 * plf] : 0.0) + (k < gc.n - 1 ? U[fo + 2 * plf] : 0.0);
      Fcv[jn] = ac * (s - 2.0 * DIM * uc);
      const long long co = b * scoarse + jn * gc.slab + off;
      Uc[co] = uc;
      Uc0[co] = uc;
      Fc[co] = Fcv[jn];
    }
    for (int jn = 0; jn < cf.sc; ++jn) {
      double If = tauf ? tauf[b * sfine + cf.map[jn] * gf.slab + fo] : 0.0;
      for (int in = 0; in < cf.sf; ++in) If += cf.dtQf[jn][in] * Ff[b * sfine + in * gf.slab + fo];
      double Ic = 0.0;
      for (int in = 0; in < cf.sc; ++in) Ic += cf.dtQc[jn][in] * Fcv[in];
      tau[b * scoarse + jn * gc.slab + off] = If - Ic;
    }
  }
}

// time interpolation of the coarse correction on the coarse grid:
// dU_m = sum_j T[m][j] (U_c,j - U_c0,j) for every fine node m (stored and combined as T)
template <typename T>
__global__ void interp_time_kernel(Grid gc, InterpCoef cf, const double *__restrict__ Uc,
                                   const double *__restrict__ Uc0, long long scoarse, T *__restrict__ dU, int batch,
                                   int m0) {
  PMG_FOR_POINTS(gc, batch) {
    PMG_POINT(gc);
    // the differences in FP64 (they cancel), the Lagrange combination in the storage
    // precision T: with FP32 storage that keeps all but 2 of the 5 FP64 operations per
    // coarse node off GB300's narrow FP64 pipe
    T d[kMaxNodes];
#pragma unroll
    for (int jn = 0; jn < kMaxNodes; ++jn) {
      if (jn >= cf.sc) break;
      const long long co = b * scoarse + jn * gc.slab + off;
      d[jn] = to_storage<T>(Uc[co] - Uc0[co]);
    }
    for (int m = m0; m < cf.sf; ++m) {
      T acc = T(0);
#pragma unroll
      for (int jn = 0; jn < kMaxNodes; ++jn)
        if (jn < cf.sc) acc += (sizeof(T) == 4 ? (T)cf.T32[m][jn] : (T)cf.T[m][jn]) * d[jn];
      dU[((long long)b * cf.sf + m) * gc.slab + off] = acc;
    }
  }
}

// coarse value at 1-based index J of one axis with odd reflection at the walls
// (J = 0 and nc+1 are the zero walls, J = -1 and nc+2 mirror J = 1 and nc)
__device__ __forceinline__ int reflect_index(int J, int nc, float *sign) {
  *sign = 1.f;
  if (J >= 1 && J <= nc) return J - 1;
  if (J == 0 || J == nc + 1) { *sign = 0.f; return 0; }
  int r = J < 0 ? -J : 2 * (nc + 1) - J;
  *sign = -1.f;
  if (r < 1 || r > nc) { *sign = 0.f; return 0; }
  return r - 1;
}

// per-axis interpolation taps of fine 0-based index i: 1-based coarse indices and
// weights (4th order (-1,9,9,-1)/16 or linear at odd points, injection at even)
__device__ __forceinline__ int interp_taps_raw(int order, int i, int *J, float *w) {
  const int i1 = i + 1;
  if ((i1 & 1) == 0) { J[0] = i1 / 2; w[0] = 1.f; return 1; }
  const int c = (i1 - 1) / 2;
  if (order == 2) { J[0] = c; J[1] = c + 1; w[0] = w[1] = 0.5f; return 2; }
  J[0] = c - 1; J[1] = c; J[2] = c + 1; J[3] = c + 2;
  w[0] = w[3] = -1.f / 16; w[1] = w[2] = 9.f / 16;
  return 4;
}

// U_f,m += I_x dU_m on a fine tile of ITX x ITY x ITZ points: the coarse box (with
// reflected wall values) is staged in shared memory and interpolated axis by axis
constexpr int ITX = 32, ITY = 8, ITZ = 8;
template <int DIM, typename T>
__global__ void __launch_bounds__(256) interp_space_kernel(Grid gf, Grid gc, int order, int sf, const T *__restrict__ dU,
                                                           double *__restrict__ Uf, long long sfine, int ntz, int m0) {
  constexpr int TY = DIM >= 2 ? ITY : 1, TZ = DIM >= 3 ? ITZ : 1;
  constexpr int CX = ITX / 2 + 4, CY = DIM >= 2 ? ITY / 2 + 4 : 1, CZ = DIM >= 3 ? ITZ / 2 + 4 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *C = (T *)smem_raw;                 // [CZ][CY][CX]
  T *X = C + CZ * CY * CX;              // [CZ][CY][ITX]
  T *Y = X + CZ * CY * ITX;             // [CZ][TY][ITX]
  const int x0 = blockIdx.x * ITX, y0 = blockIdx.y * TY;
  const int zt = blockIdx.z % ntz, b = blockIdx.z / ntz, z0 = zt * TZ;
  const int cx0 = x0 / 2 - 1, cy0 = DIM >= 2 ? y0 / 2 - 1 : 1, cz0 = DIM >= 3 ? z0 / 2 - 1 : 1;
  const int nc = gc.n, tid = threadIdx.x;
  for (int m = m0; m < sf; ++m) {
    const T *src = dU + ((long long)b * sf + m) * gc.slab;
    for (int q = tid; q < CZ * CY * CX; q += blockDim.x) {
      const int a = q % CX, bb = (q / CX) % CY, cc = q / (CX * CY);
      float sx, sy = 1.f, sz = 1.f;
      const int ix = reflect_index(cx0 + a, nc, &sx);
      const int iy = DIM >= 2 ? reflect_index(cy0 + bb, nc, &sy) : 0;
      const int iz = DIM >= 3 ? reflect_index(cz0 + cc, nc, &sz) : 0;
      const float sg = sx * sy * sz;
      C[q] = sg == 0.f ? T(0) : T(sg) * src[((long long)iz * gc.ny + iy) * gc.pitch + ix];
    }
    __syncthreads();
    for (int q = tid; q < CZ * CY * ITX; q += blockDim.x) {  // x pass
      const int x = q % ITX, row = q / ITX;
      int J[4];
      float w[4];
      const int t = interp_taps_raw(order, x0 + x, J, w);
      T acc = T(0);
      for (int u = 0; u < t; ++u) acc += T(w[u]) * C[row * CX + (J[u] - cx0)];
      X[q] = acc;
    }
    __syncthreads();
    if (DIM >= 2) {
      for (int q = tid; q < CZ * TY * ITX; q += blockDim.x) {  // y pass
        const int x = q % ITX, y = (q / ITX) % TY, zc = q / (ITX * TY);
        int J[4];
        float w[4];
        const int t = interp_taps_raw(order, y0 + y, J, w);
        T acc = T(0);
        for (int u = 0; u < t; ++u) acc += T(w[u]) * X[(zc * CY + (J[u] - cy0)) * ITX + x];
        Y[q] = acc;
      }
      __syncthreads();
    }
    const T *Src = DIM >= 2 ? Y : X;
    double *dst = Uf + (long long)b * sfine + (long long)m * gf.slab;
    for (int q = tid; q < TZ * TY * ITX; q += blockDim.x) {  // z pass and update
      const int x = q % ITX, y = (q / ITX) % TY, z = q / (ITX * TY);
      const int i = x0 + x, j = y0 + y, k = z0 + z;
      if (i >= gf.n || (DIM >= 2 && j >= gf.n) || (DIM >= 3 && k >= gf.n)) continue;
      T v;
      if (DIM >= 3) {
        int J[4];
        float w[4];
        const int t = interp_taps_raw(order, k, J, w);
        v = T(0);
        for (int u = 0; u < t; ++u) v += T(w[u]) * Src[((J[u] - cz0) * TY + y) * ITX + x];
      } else {
        v = Src[y * ITX + x];
      }
      dst[((long long)(DIM >= 3 ? k : 0) * gf.ny + (DIM >= 2 ? j : 0)) * gf.pitch + i] += to_f64(v);
    }
    __syncthreads();
  }
}

// The 3D interpolation with the thread mapping fixed: 256 threads = 32 (x) x 8 (y), and
// every tile origin even, so that the parity of a fine index -- injection or a 4-tap
// (2-tap) stencil -- is known from the thread's own x, y and the unrolled z loop; the
// coarse box is read without reflection arithmetic unless it touches a wall.  The same
// passes as interp_space_kernel (x, then y, then z with the FP64 update), with far fewer
// index instructions per fine point.
constexpr int I3CX = ITX / 2 + 4, I3CY = ITY / 2 + 4, I3CZ = ITZ / 2 + 4;

// taps of one axis for a local fine index t (tile origins are even): t odd -> the fine
// point sits on coarse box entry (t+1)/2 + 1 (injection); t even -> between box entries
// t/2 + 1 and t/2 + 2 (ORD 2), or taps t/2 .. t/2 + 3 (ORD 4)
template <typename T, int ORD>
__device__ __forceinline__ T interp3d_tap(int t, const T *src, int stride) {
  if (t & 1) return src[((t + 1) / 2 + 1) * stride];
  const int c = t / 2;
  if (ORD == 2) return T(0.5) * (src[(c + 1) * stride] + src[(c + 2) * stride]);
  return T(-1.0 / 16) * (src[c * stride] + src[(c + 3) * stride]) +
         T(9.0 / 16) * (src[(c + 1) * stride] + src[(c + 2) * stride]);
}

// coarse box entry (a, bb, cc) of the tile with 1-based box origin (cx0, cy0, cz0): the
// coarse value with odd reflection at the walls (zero on the walls themselves)
template <typename T>
__device__ __forceinline__ T interp3d_box_value(const T *__restrict__ src, const Grid &gc, int cx0, int cy0, int cz0,
                                                int a, int bb, int cc) {
  float sx, sy, sz;
  const int ix = reflect_index(cx0 + a, gc.n, &sx);
  const int iy = reflect_index(cy0 + bb, gc.n, &sy);
  const int iz = reflect_index(cz0 + cc, gc.n, &sz);
  const float sg = sx * sy * sz;
  return sg == 0.f ? T(0) : T(sg) * src[((long long)iz * gc.ny + iy) * gc.pitch + ix];
}

// whether the coarse box of a tile lies inside the grid (no reflection needed)
__device__ __forceinline__ bool interp3d_inside(int cx0, int cy0, int cz0, int nc) {
  return cx0 >= 1 && cx0 + I3CX - 1 <= nc && cy0 >= 1 && cy0 + I3CY - 1 <= nc && cz0 >= 1 && cz0 + I3CZ - 1 <= nc;
}

// x pass from the staged coarse box (rows of CS entries, box entry 0 at column C0) into
// X; the y pass from X into Y (after a barrier; Y is complete after the next barrier)
template <typename T, int ORD, int CS, int C0>
__device__ __forceinline__ void interp3d_x_pass(const T *C, T *X) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int r = ty; r < I3CZ * I3CY; r += 8) X[r * ITX + tx] = interp3d_tap<T, ORD>(tx, C + r * CS + C0, 1);
}

template <typename T, int ORD>
__device__ __forceinline__ void interp3d_y_pass(const T *X, T *Y) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int zc = 0; zc < I3CZ; ++zc) Y[(zc * ITY + ty) * ITX + tx] = interp3d_tap<T, ORD>(ty, X + zc * I3CY * ITX + tx, ITX);
}

// the coarse box of a fine tile staged in C by the threads, then the x and y passes
template <typename T, int ORD>
__device__ __forceinline__ void interp3d_xy(const T *__restrict__ src, const Grid &gc, int x0, int y0, int z0, T *C,
                                            T *X, T *Y) {
  const int cx0 = x0 / 2 - 1, cy0 = y0 / 2 - 1, cz0 = z0 / 2 - 1;  // 1-based coarse index of box entry 0
  if (interp3d_inside(cx0, cy0, cz0, gc.n)) {
    for (int q = threadIdx.x; q < I3CZ * I3CY * I3CX; q += 256) {
      const int a = q % I3CX, bb = (q / I3CX) % I3CY, cc = q / (I3CX * I3CY);
      C[q] = src[((long long)(cz0 + cc - 1) * gc.ny + (cy0 + bb - 1)) * gc.pitch + (cx0 + a - 1)];
    }
  } else {
    for (int q = threadIdx.x; q < I3CZ * I3CY * I3CX; q += 256) {
      const int a = q % I3CX, bb = (q / I3CX) % I3CY, cc = q / (I3CX * I3CY);
      C[q] = interp3d_box_value(src, gc, cx0, cy0, cz0, a, bb, cc);
    }
  }
  __syncthreads();
  interp3d_x_pass<T, ORD, I3CX, 0>(C, X);
  __syncthreads();
  interp3d_y_pass<T, ORD>(X, Y);
}

template <typename T, int ORD>
__global__ void __launch_bounds__(256) interp_space3d_kernel(Grid gf, Grid gc, int sf, const T *__restrict__ dU,
                                                             double *__restrict__ Uf, long long sfine, int ntz,
                                                             int m0) {
  __shared__ T C[I3CZ * I3CY * I3CX];
  __shared__ T X[I3CZ * I3CY * ITX];
  __shared__ T Y[I3CZ * ITY * ITX];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int x0 = blockIdx.x * ITX, y0 = blockIdx.y * ITY;
  const int zt = blockIdx.z % ntz, b = blockIdx.z / ntz, z0 = zt * ITZ;
  const int i = x0 + tx, j = y0 + ty;
  const bool mine = i < gf.n && j < gf.n;
  const long long plane = (long long)gf.ny * gf.pitch;
  for (int m = m0; m < sf; ++m) {
    const T *src = dU + ((long long)b * sf + m) * gc.slab;
    double *dst = Uf + (long long)b * sfine + (long long)m * gf.slab + (long long)j * gf.pitch + i;
    // this thread's fine column, loaded before the staging so that its HBM latency
    // overlaps the shared-memory passes
    double uold[ITZ];
#pragma unroll
    for (int z = 0; z < ITZ; ++z) uold[z] = mine && z0 + z < gf.n ? dst[(z0 + z) * plane] : 0.0;
    interp3d_xy<T, ORD>(src, gc, x0, y0, z0, C, X, Y);
    __syncthreads();
    if (mine) {
#pragma unroll
      for (int z = 0; z < ITZ; ++z) {  // z pass and the FP64 update
        const int k = z0 + z;
        if (k < gf.n) {
          const T dv = interp3d_tap<T, ORD>(z, Y + ty * ITX + tx, ITY * ITX);
          if constexpr (sizeof(T) == 4) dst[k * plane] = uold[z] + widen_exact(dv);
          else dst[k * plane] = uold[z] + dv;
        }
      }
    }
    __syncthreads();
  }
}

// The same interpolation with every global access done by TMA: the FP64 32 x 8 x 8 fine
// tile of node m+1 is loaded (cp.async.bulk.tensor, one elected thread) while node m is
// interpolated, the coarse box of node m+1 as soon as the x pass of node m has consumed
// the box buffer, the z pass adds the correction to the staged fine tile in place, and
// the tile goes back by a TMA bulk store.  Rows and planes past the fine grid arrive as
// zeros and are clipped from the store; the pad column is written back as it was read.
// The coarse box is loaded 24 entries wide from the 4-aligned x index x0/2 - 4 (the TMA
// x coordinate must be 16-byte aligned), so box entry 0 is column 2; entries outside the
// coarse grid arrive as zeros and, in tiles at a wall, are then overwritten with their
// reflected values by the threads.  Two fine-tile buffers: a buffer is refilled only
// after the bulk store of its previous node has read it out.  Same arithmetic as
// interp_space3d_kernel, so the results are bitwise equal.
constexpr int I3CW = I3CX + 4;  // staged coarse row: 4-aligned start, multiple of 16 bytes

template <typename T, int ORD>
__global__ void __launch_bounds__(256) interp_space3d_tma_kernel(const __grid_constant__ CUtensorMap tmu,
                                                                 const __grid_constant__ CUtensorMap tmc, Grid gf,
                                                                 Grid gc, int sf, const T *__restrict__ dU, int ntz,
                                                                 int m0) {
  using namespace tma;
  constexpr uint32_t UB = ITX * ITY * ITZ * 8;                 // bytes of one FP64 fine tile
  constexpr uint32_t CB = I3CZ * I3CY * I3CW * sizeof(T);      // bytes of one coarse box
  extern __shared__ __align__(1024) unsigned char sm[];
  double(*Ut)[ITZ][ITY][ITX] = (double(*)[ITZ][ITY][ITX])sm;  // [2]
  T *C = (T *)(sm + 2 * UB);                                    // [I3CZ][I3CY][I3CW]
  T *X = C + I3CZ * I3CY * I3CW;
  T *Y = X + I3CZ * I3CY * ITX;
  uint64_t *bar = (uint64_t *)(Y + I3CZ * ITY * ITX);  // [3]: fine tiles 0, 1; coarse box
  int *s_bad = (int *)(bar + 3);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int x0 = blockIdx.x * ITX, y0 = blockIdx.y * ITY;
  const int zt = blockIdx.z % ntz, b = blockIdx.z / ntz, z0 = zt * ITZ;
  const int cx0 = x0 / 2 - 1, cy0 = y0 / 2 - 1, cz0 = z0 / 2 - 1;  // 1-based coarse index of box entry 0
  const bool inside = interp3d_inside(cx0, cy0, cz0, gc.n);
  const int i = x0 + tx, j = y0 + ty;
  const bool mine = i < gf.n && j < gf.n;
  auto load_c = [&](int m) {
    mbar_expect_tx(&bar[2], CB);
    tma_load_4d(C, &tmc, x0 / 2 - 4, cy0 - 1, cz0 - 1, b * sf + m, &bar[2]);
  };
  if (threadIdx.x == 0) {
    for (int q = 0; q < 3; ++q) mbar_init(&bar[q]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_proxy_async_smem();
    *s_bad = 0;
    mbar_expect_tx(&bar[0], UB);
    tma_load_4d(&Ut[0][0][0][0], &tmu, x0, y0, z0, b * sf + m0, &bar[0]);
    load_c(m0);
  }
  __syncthreads();
  int issued = m0, issued_c = 1;  // thread 0: last node whose fine tile load was issued; box loads issued
  for (int m = m0; m < sf; ++m) {
    const int t = m - m0, buf = t & 1;
    if (threadIdx.x == 0 && m + 1 < sf) {
      bulk_wait_read_all();  // the store of node m-1 has read buffer buf^1 out
      mbar_expect_tx(&bar[buf ^ 1], UB);
      tma_load_4d(&Ut[buf ^ 1][0][0][0], &tmu, x0, y0, z0, b * sf + m + 1, &bar[buf ^ 1]);
      issued = m + 1;
    }
    bool ok = mbar_wait(&bar[2], (uint32_t)t & 1u);  // the t-th coarse box: phase t
    if (ok && !inside) {  // reflected values where the box crosses a wall
      const T *src = dU + ((long long)b * sf + m) * gc.slab;
      for (int q = threadIdx.x; q < I3CZ * I3CY * I3CX; q += 256) {
        const int a = q % I3CX, bb = (q / I3CX) % I3CY, cc = q / (I3CX * I3CY);
        const int J = cx0 + a, K = cy0 + bb, L = cz0 + cc;
        if (J < 1 || J > gc.n || K < 1 || K > gc.n || L < 1 || L > gc.n)
          C[(cc * I3CY + bb) * I3CW + a + 2] = interp3d_box_value(src, gc, cx0, cy0, cz0, a, bb, cc);
      }
      fence_proxy_async_smem();  // these writes precede the next box's TMA load
    }
    if (!ok) *s_bad = 1;
    __syncthreads();
    if (*s_bad) break;  // uniform: read after the barrier
    interp3d_x_pass<T, ORD, I3CW, 2>(C, X);
    __syncthreads();
    if (threadIdx.x == 0 && m + 1 < sf) {  // the box buffer is free again
      load_c(m + 1);
      ++issued_c;
    }
    interp3d_y_pass<T, ORD>(X, Y);
    ok = mbar_wait(&bar[buf], (uint32_t)(t >> 1) & 1u);  // the j-th load into a buffer: phase j
    if (!ok) *s_bad = 1;
    __syncthreads();
    if (*s_bad) break;
    if (mine) {
#pragma unroll
      for (int z = 0; z < ITZ; ++z) {  // z pass and the FP64 update, in the staged tile
        if (z0 + z < gf.n) {
          const T dv = interp3d_tap<T, ORD>(z, Y + ty * ITX + tx, ITY * ITX);
          if constexpr (sizeof(T) == 4) Ut[buf][z][ty][tx] = Ut[buf][z][ty][tx] + widen_exact(dv);
          else Ut[buf][z][ty][tx] = Ut[buf][z][ty][tx] + dv;
        }
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tma_store_4d(&tmu, &Ut[buf][0][0][0], x0, y0, z0, b * sf + m);
      bulk_commit();
    }
  }
  if (threadIdx.x == 0) {
    if (*s_bad) {
      atomicExch(&g_interp_timeout, 1);
      // loads possibly still in flight: the last two fine tiles (one per buffer, phases as
      // numbered above) and the last coarse box; wait for them (bounded) before the CTA's
      // shared memory is released
      for (int t = issued - m0 - 1; t <= issued - m0; ++t)
        if (t >= 0) mbar_wait(&bar[t & 1], (uint32_t)(t >> 1) & 1u);
      mbar_wait(&bar[2], (uint32_t)(issued_c - 1) & 1u);
    }
    bulk_wait_all();  // every bulk store complete before the CTA exits
  }
}

// self-check of narrow_rn against the hardware conversion on generated bit patterns:
// a quarter uniform over all doubles, the rest steered into the float range around
// subnormals and overflow, onto exact ties and onto exactly representable values
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ULL;
  x ^= x >> 33;
  return x;
}

__global__ void narrow_check_kernel(long long count, unsigned long long seed, unsigned long long *bad) {
  unsigned long long nbad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long bits = mix64(seed + (unsigned long long)i);
    const unsigned sel = (unsigned)(i & 3);
    if (sel != 0) {
      const unsigned long long ex = 1023 - 160 + mix64(seed ^ (unsigned long long)(3 * i + 1)) % 300;
      bits = (bits & 0x800fffffffffffffULL) | (ex << 52);
      if (sel == 2) bits = (bits & ~0xfffffffULL) | 0x10000000ULL;  // a tie at the float rounding position
      if (sel == 3 && (i & 4)) bits &= ~0x1fffffffULL;              // representable when normal
    }
    const double v = __longlong_as_double((long long)bits);
    const float hw = __double2float_rn(v), sw = narrow_rn(v);
    if (v != v ? !(sw != sw) : __float_as_uint(hw) != __float_as_uint(sw)) ++nbad;
  }
  if (nbad) atomicAdd(bad, nbad);
}

// every float bit pattern once: widen_exact against the hardware conversion
__global__ void widen_check_kernel(unsigned long long *bad) {
  unsigned long long nbad = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < (1ULL << 32);
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const float f = __uint_as_float((unsigned)i);
    const double hw = (double)f, sw = widen_exact(f);
    if (f != f ? !(sw != sw) : __double_as_longlong(hw) != __double_as_longlong(sw)) ++nbad;
  }
  if (nbad) atomicAdd(bad, nbad);
}

__global__ void colloc_residual_kernel(Grid g, ResCoef cf, const double *__restrict__ U, const double *__restrict__ F,
                                       long long stride, int batch, unsigned long long *out) {
  for (int zb = blockIdx.z; zb < g.nz * batch; zb += gridDim.z) {
    const int k = zb % g.nz, b = zb / g.nz;
    double mx = 0.0;
    for (int j = blockIdx.y * blockDim.y + threadIdx.y; j < g.ny; j += gridDim.y * blockDim.y)
      for (int i = threadIdx.x; i < g.n; i += blockDim.x) {
        const long long off = ((long long)k * g.ny + j) * g.pitch + i;
        double Fv[kMaxNodes];
        for (int in = 0; in < cf.s; ++in) Fv[in] = F[b * stride + in * g.slab + off];
        const double u0 = U[b * stride + off];
        for (int m = 1; m < cf.s; ++m) {
          double v = u0;
          for (int in = 0; in < cf.s; ++in) v += cf.dtQ[m][in] * Fv[in];
          v -= U[b * stride + m * g.slab + off];
          const double av = fabs(v);
          if (!(av <= mx)) mx = av;
        }
      }
    warp_max_atomic(mx, out + b);
  }
}

// End-of-iteration pass of the fine level (fixed V-cycle counts): from U alone,
//   F_j = nu Lap_h U_j at every node (not stored),
//   q_m = sum_j dt (Q[m+1][j] - Q[m][j]) F_j - U_{m+1} (the node-to-node quadrature S F
//   of Eq. sdc-be minus the current iterate): u_m + q_m is the initial residual of
//   sub-step m of the next sweep (Eq. SDCcompactLIII with initial guess u^k_{m+1}),
//   collocation residual r_m = U_0 + dt sum_j Q[m][j] F_j - U_m (Eq. resid), max-reduced
//   per slice, from the same q's: r_1 = U_0 + q_0, r_{m+1} = r_m + q_m + U_m (the rows of
//   Q are the partial sums of the rows of S).
// One FMA chain per q (started from -U_{m+1}) and two adds per residual: 51 FP64
// instructions per slice-point for 5 nodes instead of 55 with the cumulative rows.
// cf.dS holds (nu / h^2) dt S here (scaled by the launcher).  S = number of nodes, a
// compile-time constant so that no predicated-off FP64 work is issued; O4 = the
// fourth-order stencil.
template <int DIM, int S, bool O4>
__global__ void fine_rhs_residual_kernel(Grid g, ResCoef cf, const double *__restrict__ U, long long stride,
                                         double *__restrict__ q, long long sq, int batch, unsigned long long *res) {
  for (int zb = blockIdx.z; zb < g.nz * batch; zb += gridDim.z) {
    const int k = zb % g.nz, b = zb / g.nz;
    unsigned long long mxb = 0ULL;
    for (int j = blockIdx.y * blockDim.y + threadIdx.y; j < g.ny; j += gridDim.y * blockDim.y)
      for (int i = threadIdx.x; i < g.n; i += blockDim.x) {
        const long long off = ((long long)k * g.ny + j) * g.pitch + i;
        const double *Ub = U + b * stride;
        // G_j = h^2 Lap_h U_j; the factor nu / h^2 is folded into the weights (aQ = a dtQ)
        double Uv[S], Gv[S];
#pragma unroll
        for (int jn = 0; jn < S; ++jn) {
          const double *Uj = Ub + jn * g.slab;
          Uv[jn] = Uj[off];
          Gv[jn] = O4 ? lap4_h2<DIM>(Uj, g, i, j, k, off) : nbsum<DIM>(Uj, g, i, j, k, off) - 2.0 * DIM * Uv[jn];
        }
        double r = 0.0;
#pragma unroll
        for (int m = 0; m + 1 < S; ++m) {
          double qm = -Uv[m + 1];
#pragma unroll
          for (int jn = 0; jn < S; ++jn) qm = fma(cf.dS[m][jn], Gv[jn], qm);
          q[b * sq + m * g.slab + off] = qm;
          r = m == 0 ? Uv[0] + qm : r + (qm + Uv[m]);  // r_{m+1}
          // |r| as a bit pattern: for non-negative doubles (and NaN above Inf) the
          // unsigned integer order is the numeric order, so no FP64 compare is issued
          const unsigned long long rb = (unsigned long long)__double_as_longlong(r) & 0x7fffffffffffffffULL;
          mxb = rb > mxb ? rb : mxb;
        }
      }
    if (res) {
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, mxb, o);
        mxb = w > mxb ? w : mxb;
      }
      if ((threadIdx.x & 31) == 0 && mxb != 0ULL) atomicMax(res + b, mxb);
    }
  }
}

// The same pass when U[b][0] is a copy of U[b-1][S-1] for every slice b >= 1 (right after
// the send-forward): one thread walks all slices of its grid point and takes node 0's
// value and Laplacian from the previous slice's last node -- bitwise the same numbers,
// one FP64 Laplacian and 7 loads fewer per slice-point.  Per-slice residual maxima are
// reduced per warp into shared memory, then once per CTA into res.  The loop bound is
// rounded up to whole warps so that every lane takes part in the shuffles.
template <int DIM, int S>
__global__ void __launch_bounds__(256, 4) fine_rhs_chain_kernel(Grid g, ResCoef cf, const double *__restrict__ U,
                                                             long long stride, double *__restrict__ q, long long sq,
                                                             int batch, unsigned long long *res) {
  extern __shared__ unsigned long long smax[];  // [batch]
  for (int b = threadIdx.x; b < batch; b += blockDim.x) smax[b] = 0ULL;
  __syncthreads();
  const long long total = (long long)g.nz * g.ny * g.pitch, tot32 = (total + 31) & ~31LL;
  const int lane = threadIdx.x & 31;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < tot32;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % g.pitch);
    const long long rest = p / g.pitch;
    const int j = (int)(rest % g.ny), k = (int)(rest / g.ny);
    const bool valid = p < total && i < g.n;
    const long long off = valid ? p : 0;
    double Ulast = 0.0, Glast = 0.0;
    for (int b = 0; b < batch; ++b) {
      unsigned long long mxb = 0ULL;
      if (valid) {
        const double *Ub = U + b * stride;
        double Uv[S], Gv[S];
        if (b == 0) {
          Uv[0] = Ub[off];
          Gv[0] = nbsum<DIM>(Ub, g, i, j, k, off) - 2.0 * DIM * Uv[0];
        } else {
          Uv[0] = Ulast;
          Gv[0] = Glast;
        }
#pragma unroll
        for (int jn = 1; jn < S; ++jn) {
          const double *Uj = Ub + jn * g.slab;
          Uv[jn] = Uj[off];
          Gv[jn] = nbsum<DIM>(Uj, g, i, j, k, off) - 2.0 * DIM * Uv[jn];
        }
        double r = 0.0;
#pragma unroll
        for (int m = 0; m + 1 < S; ++m) {
          double qm = -Uv[m + 1];
#pragma unroll
          for (int jn = 0; jn < S; ++jn) qm = fma(cf.dS[m][jn], Gv[jn], qm);
          q[b * sq + m * g.slab + off] = qm;
          r = m == 0 ? Uv[0] + qm : r + (qm + Uv[m]);  // r_{m+1}
          const unsigned long long rb = (unsigned long long)__double_as_longlong(r) & 0x7fffffffffffffffULL;
          mxb = rb > mxb ? rb : mxb;
        }
        Ulast = Uv[S - 1];
        Glast = Gv[S - 1];
      }
      if (res) {
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long w = __shfl_xor_sync(0xffffffffu, mxb, o);
          mxb = w > mxb ? w : mxb;
        }
        if (lane == 0 && mxb != 0ULL) atomicMax(&smax[b], mxb);
      }
    }
  }
  __syncthreads();
  if (res)
    for (int b = threadIdx.x; b < batch; b += blockDim.x)
      if (smax[b] != 0ULL) atomicMax(res + b, smax[b]);
}

// FAS restriction with the fine F evaluated from U_f at the coarse points only.  cf.dtQf
// holds (nu / h_f^2) dt Q_fine here (scaled by the launcher), so the fine Laplacians enter
// unscaled; a coarse node whose quadrature rows are zero (t = 0) gets tau = 0 directly.
template <int DIM, int SF, int SC>
__global__ void fas_restrict_u_kernel(Grid gf, Grid gc, FASCoef cf, const double *__restrict__ Uf, long long sfine,
                                      double *__restrict__ Uc, double *__restrict__ Fc, double *__restrict__ tau,
                                      double *__restrict__ Uc0, long long scoarse, int batch) {
  const double ac = cf.nu * gc.ih2;
  const long long plf = (long long)gf.ny * gf.pitch;
  PMG_FOR_POINTS(gc, batch) {
    PMG_POINT(gc);
    const int fi = 2 * i + 1, fj = DIM >= 2 ? 2 * j + 1 : 0, fk = DIM >= 3 ? 2 * k + 1 : 0;
    const long long fo = ((long long)fk * gf.ny + fj) * gf.pitch + fi;
    constexpr int NF = SF ? SF : kMaxNodes, NC = SC ? SC : kMaxNodes;  // 0: counts known at run time
    double Fcv[NC], Ffv[NF];
#pragma unroll
    for (int in = 0; in < NF; ++in) {
      if (SF == 0 && in >= cf.sf) break;
      const double *U = Uf + b * sfine + in * gf.slab;
      Ffv[in] = lap_h2<DIM>(U, gf, fi, fj, fk, fo);  // h_f^2 Lap_h U (nu / h_f^2 is in dtQf)
    }
#pragma unroll
    for (int jn = 0; jn < NC; ++jn) {
      if (SC == 0 && jn >= cf.sc) break;
      const double *U = Uf + b * sfine + cf.map[jn] * gf.slab;
      const double uc = U[fo];
      double s = (i > 0 ? U[fo - 2] : 0.0) + (i < gc.n - 1 ? U[fo + 2] : 0.0);
      if (DIM >= 2) s += (j > 0 ? U[fo - 2 * gf.pitch] : 0.0) + (j < gc.n - 1 ? U[fo + 2 * gf.pitch] : 0.0);
      if (DIM >= 3) s += (k > 0 ? U[fo - 2 * plf] : 0.0) + (k < gc.n - 1 ? U[fo + 2 * plf] : 0.0);
      Fcv[jn] = ac * (s - 2.0 * DIM * uc);
      const long long co = b * scoarse + jn * gc.slab + off;
      Uc[co] = uc;
      Uc0[co] = uc;
      Fc[co] = Fcv[jn];
    }
#pragma unroll
    for (int jn = 0; jn < NC; ++jn) {
      if (SC == 0 && jn >= cf.sc) break;
      if (cf.zero_rows & (1 << jn)) {  // uniform over the launch
        tau[b * scoarse + jn * gc.slab + off] = 0.0;
        continue;
      }
      double If = 0.0;
#pragma unroll
      for (int in = 0; in < NF; ++in)
        if (SF != 0 || in < cf.sf) If += cf.dtQf[jn][in] * Ffv[in];
      double Ic = 0.0;
#pragma unroll
      for (int in = 0; in < NC; ++in)
        if (SC != 0 || in < cf.sc) Ic += cf.dtQc[jn][in] * Fcv[in];
      tau[b * scoarse + jn * gc.slab + off] = If - Ic;
    }
  }
}

// Pointwise kernels over whole padded slabs: blockIdx.y selects the grid of the batch and
// the x blocks stride over its slab two elements at a time.  The pitch n + 1 is a power
// of two, so every slab and stride is even and a pair never straddles rows; the pair
// that ends a row holds the last interior point and the pad, and the pad is written as
// zero.  Few long-lived blocks instead of one block per row.
template <typename T>
__global__ void resid_pt_flat_kernel(long long slab, int pitch, const double *__restrict__ um, long long sum,
                                     const double *__restrict__ qm, long long sq, T *__restrict__ f) {
  const int b = blockIdx.y;
  const double2 *U = (const double2 *)(um + b * sum), *Q = (const double2 *)(qm + b * sq);
  const long long n2 = slab / 2;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n2; p += (long long)gridDim.x * blockDim.x) {
    const double2 u = U[p], q = Q[p];
    const bool padpair = (((unsigned)(2 * p)) & (unsigned)(pitch - 1)) == (unsigned)(pitch - 2);
    if constexpr (sizeof(T) == 4) {
      ((float2 *)(f + b * slab))[p] = make_float2(narrow_rn(u.x + q.x), padpair ? 0.f : narrow_rn(u.y + q.y));
    } else {
      ((double2 *)(f + b * slab))[p] = make_double2(u.x + q.x, padpair ? 0.0 : u.y + q.y);
    }
  }
}

__global__ void copy_flat_kernel(long long slab, int pitch, const double *__restrict__ src, long long ss,
                                 double *__restrict__ dst, long long sd) {
  const int b = blockIdx.y;
  const double2 *S = (const double2 *)(src + b * ss);
  double2 *D = (double2 *)(dst + b * sd);
  const long long n2 = slab / 2;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n2; p += (long long)gridDim.x * blockDim.x) {
    double2 v = S[p];
    if ((((unsigned)(2 * p)) & (unsigned)(pitch - 1)) == (unsigned)(pitch - 2)) v.y = 0.0;
    D[p] = v;
  }
}

// the flat kernels need a power-of-two pitch, even strides and slab positions that fit
// 32 bits (the pad test), and at most 65535 grids
bool flat_ok(const Grid &g, int batch, long long strides) {
  return batch <= 65535 && (g.pitch & (g.pitch - 1)) == 0 && ((strides | g.slab) & 1) == 0 && g.slab < (1LL << 31);
}

// x blocks per grid for the flat kernels: about 8 blocks of 256 per SM in total
dim3 flat_grid(long long slab, int batch) {
  long long gx = (152LL * 8 + batch - 1) / batch, need = (slab / 2 + 255) / 256;
  if (gx > need) gx = need;
  if (gx < 1) gx = 1;
  return dim3((unsigned)gx, (unsigned)batch, 1);
}

__global__ void copy_kernel(Grid g, const double *__restrict__ src, long long ss, double *__restrict__ dst,
                            long long sd, int batch) {
  PMG_FOR_POINTS(g, batch) {
    PMG_POINT(g);
    dst[b * sd + off] = src[b * ss + off];
  }
}

__global__ void pack_kernel(Grid g, const double *__restrict__ dense, long long sdense, double *__restrict__ pad,
                            long long spad, int batch) {
  PMG_FOR_POINTS(g, batch) {
    PMG_POINT(g);
    const long long dn = ((long long)k * g.ny + j) * g.n + i;
    pad[b * spad + off] = dense[b * sdense + dn];
  }
}

__global__ void unpack_kernel(Grid g, const double *__restrict__ pad, long long spad, double *__restrict__ dense,
                              long long sdense, int batch) {
  PMG_FOR_POINTS(g, batch) {
    PMG_POINT(g);
    const long long dn = ((long long)k * g.ny + j) * g.n + i;
    dense[b * sdense + dn] = pad[b * spad + off];
  }
}

}  // namespace

// ------------------------------------------------------------------ launchers

#define PMG_DIM_SWITCH(dim, CALL) \
  switch (dim) {                  \
    case 1: { constexpr int D = 1; CALL; } break; \
    case 2: { constexpr int D = 2; CALL; } break; \
    default: { constexpr int D = 3; CALL; } break; \
  }

cudaError_t k_residual0(const Launch &L, const Grid &g, double c, Prec pr, const double *um, long long sum,
                        const double *qm, long long sq, const double *u1, long long s1, void *f, int batch,
                        unsigned long long *rnorm, unsigned long long *bnorm) {
  dim3 gr, bl;
  config(g, batch, gr, bl);
  Scope sc(L, K_RESIDUAL0, g, batch, pr);
  if (pr == F64)
    PMG_DIM_SWITCH(g.dim, (residual0_kernel<D, double><<<gr, bl, 0, L.stream>>>(
                              g, c, um, sum, qm, sq, u1, s1, (double *)f, batch, rnorm, bnorm)))
  else
    PMG_DIM_SWITCH(g.dim, (residual0_kernel<D, float><<<gr, bl, 0, L.stream>>>(
                              g, c, um, sum, qm, sq, u1, s1, (float *)f, batch, rnorm, bnorm)))
  return sc.done();
}

cudaError_t k_smooth_jacobi(const Launch &L, const Grid &g, double c, double omega, Prec pr, const void *ein,
                            void *eout, const void *f, int batch, bool first, int threads) {
  dim3 gr, bl;
  config(g, batch, gr, bl, threads);
  Scope sc(L, K_JACOBI, g, batch, pr);
  if (pr == F64)
    PMG_DIM_SWITCH(g.dim, (jacobi_kernel<D, double><<<gr, bl, 0, L.stream>>>(
                              g, c, omega, (const double *)ein, (double *)eout, (const double *)f, batch, first)))
  else
    PMG_DIM_SWITCH(g.dim, (jacobi_kernel<D, float><<<gr, bl, 0, L.stream>>>(
                              g, (float)c, (float)omega, (const float *)ein, (float *)eout, (const float *)f, batch,
                              first)))
  return sc.done();
}

cudaError_t k_smooth_rbgs(const Launch &L, const Grid &g, double c, double omega, Prec pr, void *e, const void *f,
                          int batch, int colour, bool first, int threads) {
  dim3 gr, bl;
  config(g, batch, gr, bl, threads);
  Scope sc(L, K_RBGS, g, batch, pr);
  if (pr == F64)
    PMG_DIM_SWITCH(g.dim, (rbgs_kernel<D, double><<<gr, bl, 0, L.stream>>>(g, c, omega, (double *)e,
                                                                               (const double *)f, batch, colour, first)))
  else
    PMG_DIM_SWITCH(g.dim, (rbgs_kernel<D, float><<<gr, bl, 0, L.stream>>>(g, (float)c, (float)omega, (float *)e,
                                                                              (const float *)f, batch, colour, first)))
  return sc.done();
}

cudaError_t k_residual_restrict(const Launch &L, const Grid &gf, const Grid &gc, double c, Prec pr, const void *e,
                                const void *f, void *fc, int batch) {
  dim3 gr, bl;
  config(gc, batch, gr, bl);
  Scope sc(L, K_RESRESTRICT, gc, batch, pr);
  if (pr == F64)
    PMG_DIM_SWITCH(gf.dim, (resrestrict_kernel<D, double><<<gr, bl, 0, L.stream>>>(
                               gf, gc, c, (const double *)e, (const double *)f, (double *)fc, batch)))
  else
    PMG_DIM_SWITCH(gf.dim, (resrestrict_kernel<D, float><<<gr, bl, 0, L.stream>>>(
                               gf, gc, (float)c, (const float *)e, (const float *)f, (float *)fc, batch)))
  return sc.done();
}

cudaError_t k_prolong_add(const Launch &L, const Grid &gf, const Grid &gc, Prec pr, const void *ec, void *e,
                          int batch) {
  dim3 gr, bl;
  config(gf, batch, gr, bl);
  Scope sc(L, K_PROLONG, gf, batch, pr);
  if (pr == F64)
    PMG_DIM_SWITCH(gf.dim,
                   (prolong_kernel<D, double><<<gr, bl, 0, L.stream>>>(gf, gc, (const double *)ec, (double *)e, batch)))
  else
    PMG_DIM_SWITCH(gf.dim,
                   (prolong_kernel<D, float><<<gr, bl, 0, L.stream>>>(gf, gc, (const float *)ec, (float *)e, batch)))
  return sc.done();
}

cudaError_t k_coarse_solve(const Launch &L, const Grid &g3, Prec pr, const void *minv, const void *f, void *e,
                           int batch) {
  dim3 gr, bl;
  config(g3, batch, gr, bl);
  Scope sc(L, K_COARSE, g3, batch, pr);
  if (pr == F64)
    PMG_DIM_SWITCH(g3.dim, (coarse_solve_kernel<D, double><<<gr, bl, 0, L.stream>>>(
                               g3, (const double *)minv, (const double *)f, (double *)e, batch)))
  else
    PMG_DIM_SWITCH(g3.dim, (coarse_solve_kernel<D, float><<<gr, bl, 0, L.stream>>>(
                               g3, (const float *)minv, (const float *)f, (float *)e, batch)))
  return sc.done();
}

cudaError_t k_update_u(const Launch &L, const Grid &g, Prec pr, double *u, long long su, const void *e, int batch,
                       const int *active) {
  dim3 gr, bl;
  config(g, batch, gr, bl);
  Scope sc(L, K_UPDATE, g, batch, pr);
  if (pr == F64)
    update_u_kernel<double><<<gr, bl, 0, L.stream>>>(g, u, su, (const double *)e, batch, active);
  else
    update_u_kernel<float><<<gr, bl, 0, L.stream>>>(g, u, su, (const float *)e, batch, active);
  return sc.done();
}

cudaError_t k_zero(const Launch &L, const Grid &g, Prec pr, void *e, int batch) {
  dim3 gr, bl;
  config(g, batch, gr, bl);
  Scope sc(L, K_ZERO, g, batch, pr);
  if (pr == F64)
    zero_kernel<double><<<gr, bl, 0, L.stream>>>(g, (double *)e, batch);
  else
    zero_kernel<float><<<gr, bl, 0, L.stream>>>(g, (float *)e, batch);
  return sc.done();
}

cudaError_t k_apply_A(const Launch &L, const Grid &g, double nu, const double *u, long long su, double *F,
                      long long sF, int batch) {
  dim3 gr, bl;
  config(g, batch, gr, bl);
  Scope sc(L, K_APPLY_A, g, batch, 0);
  PMG_DIM_SWITCH(g.dim, (apply_A_kernel<D><<<gr, bl, 0, L.stream>>>(g, nu, u, su, F, sF, batch)))
  return sc.done();
}

cudaError_t k_resid_pt(const Launch &L, const Grid &g, Prec pr, const double *um, long long sum, const double *qm,
                       long long sq, void *f, int batch) {
  Scope sc(L, K_RESID_PT, g, batch, pr);
  if (flat_ok(g, batch, sum | sq)) {
    const dim3 gr = flat_grid(g.slab, batch);
    if (pr == F64)
      resid_pt_flat_kernel<double><<<gr, 256, 0, L.stream>>>(g.slab, g.pitch, um, sum, qm, sq, (double *)f);
    else
      resid_pt_flat_kernel<float><<<gr, 256, 0, L.stream>>>(g.slab, g.pitch, um, sum, qm, sq, (float *)f);
    return sc.done();
  }
  dim3 gr, bl;
  config(g, batch, gr, bl);
  if (pr == F64)
    resid_pt_kernel<double><<<gr, bl, 0, L.stream>>>(g, um, sum, qm, sq, (double *)f, batch);
  else
    resid_pt_kernel<float><<<gr, bl, 0, L.stream>>>(g, um, sum, qm, sq, (float *)f, batch);
  return sc.done();
}

cudaError_t k_sf_rhs(const Launch &L, const Grid &g, const SFCoef &cf, const double *F, const double *U, long long sF,
                     const double *tau, long long stau, double *q, long long sq, int batch) {
  dim3 gr, bl;
  config(g, batch, gr, bl);
  Scope sc(L, K_SF_RHS, g, batch, 0);
  switch (cf.s) {
#define PMG_SF_CASE(S) \
  case S: sf_rhs_kernel<S><<<gr, bl, 0, L.stream>>>(g, cf, F, U, sF, tau, stau, q, sq, batch); break;
    PMG_SF_CASE(2) PMG_SF_CASE(3) PMG_SF_CASE(4) PMG_SF_CASE(5) PMG_SF_CASE(6) PMG_SF_CASE(7) PMG_SF_CASE(8)
    PMG_SF_CASE(9)
#undef PMG_SF_CASE
    default: return cudaErrorInvalidValue;
  }
  return sc.done();
}

cudaError_t k_fas_restrict(const Launch &L, const Grid &gf, const Grid &gc, const FASCoef &cf, const double *Uf,
                           const double *Ff, long long sfine, double *Uc, double *Fc, double *tau, double *Uc0,
                           long long scoarse, int batch, const double *tauf) {
  dim3 gr, bl;
  config(gc, batch, gr, bl);
  Scope sc(L, K_FAS, gc, batch, 0);
  PMG_DIM_SWITCH(gf.dim, (fas_restrict_kernel<D><<<gr, bl, 0, L.stream>>>(gf, gc, cf, Uf, Ff, sfine, Uc, Fc, tau,
                                                                             Uc0, scoarse, batch, tauf)))
  return sc.done();
}

cudaError_t k_interp_time(const Launch &L, const Grid &gc, const InterpCoef &cf, Prec pr, const double *Uc,
                          const double *Uc0, long long scoarse, void *dU, int batch, int m0) {
  dim3 gr, bl;
  config(gc, batch, gr, bl);
  Scope sc(L, K_INTERP_T, gc, batch, pr);
  if (pr == F64)
    interp_time_kernel<double><<<gr, bl, 0, L.stream>>>(gc, cf, Uc, Uc0, scoarse, (double *)dU, batch, m0);
  else
    interp_time_kernel<float><<<gr, bl, 0, L.stream>>>(gc, cf, Uc, Uc0, scoarse, (float *)dU, batch, m0);
  return sc.done();
}

template <int D, typename T>
cudaError_t launch_interp_space(const Launch &L, const Grid &gf, const Grid &gc, int order, int sf, const void *dU,
                                double *Uf, long long sfine, int batch, int m0) {
  constexpr int TY = D >= 2 ? ITY : 1, TZ = D >= 3 ? ITZ : 1;
  constexpr int CX = ITX / 2 + 4, CY = D >= 2 ? ITY / 2 + 4 : 1, CZ = D >= 3 ? ITZ / 2 + 4 : 1;
  const size_t smem = sizeof(T) * (CZ * CY * CX + CZ * CY * ITX + CZ * TY * ITX);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(interp_space_kernel<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const int ntx = (gf.n + ITX - 1) / ITX, nty = (gf.ny + TY - 1) / TY, ntz = (gf.nz + TZ - 1) / TZ;
  dim3 gr(ntx, nty, ntz * batch);
  interp_space_kernel<D, T><<<gr, 256, smem, L.stream>>>(gf, gc, order, sf, (const T *)dU, Uf, sfine, ntz, m0);
  return cudaSuccess;
}

template <typename T, int ORD>
cudaError_t launch_interp_space3d_tma(const Launch &L, const Grid &gf, const Grid &gc, int sf, const void *dU,
                                      double *Uf, int batch, int m0) {
  const size_t smem = 2 * (size_t)ITX * ITY * ITZ * 8 +
                      sizeof(T) * (I3CZ * I3CY * I3CW + I3CZ * I3CY * ITX + I3CZ * ITY * ITX) + 3 * sizeof(uint64_t) +
                      sizeof(int);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(interp_space3d_tma_kernel<T, ORD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const cuuint32_t es[4] = {1, 1, 1, 1};
  // the fine grid functions of all slices and nodes as one 4D tensor (x, y, z, slice * sf + node)
  CUtensorMap mu, mc;
  const cuuint64_t dims[4] = {(cuuint64_t)gf.pitch, (cuuint64_t)gf.ny, (cuuint64_t)gf.nz, (cuuint64_t)batch * sf};
  const cuuint64_t strides[3] = {(cuuint64_t)gf.pitch * 8, (cuuint64_t)gf.ny * gf.pitch * 8, (cuuint64_t)gf.slab * 8};
  const cuuint32_t box[4] = {ITX, ITY, ITZ, 1};
  // the coarse corrections likewise, x limited to the interior (the pad column reads as zero)
  const cuuint64_t cdims[4] = {(cuuint64_t)gc.n, (cuuint64_t)gc.ny, (cuuint64_t)gc.nz, (cuuint64_t)batch * sf};
  const cuuint64_t cstrides[3] = {(cuuint64_t)gc.pitch * sizeof(T), (cuuint64_t)gc.ny * gc.pitch * sizeof(T),
                                  (cuuint64_t)gc.slab * sizeof(T)};
  const cuuint32_t cbox[4] = {I3CW, I3CY, I3CZ, 1};
  if (tma::encoder()(&mu, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, Uf, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      tma::encoder()(&mc, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                     const_cast<void *>(dU), cdims, cstrides, cbox, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int ntx = gf.pitch / ITX, nty = (gf.n + ITY - 1) / ITY, ntz = (gf.n + ITZ - 1) / ITZ;
  dim3 gr(ntx, nty, ntz * batch);
  interp_space3d_tma_kernel<T, ORD><<<gr, 256, smem, L.stream>>>(mu, mc, gf, gc, sf, (const T *)dU, ntz, m0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_interp_space3d(const Launch &L, const Grid &gf, const Grid &gc, int order, int sf, const void *dU,
                                  double *Uf, long long sfine, int batch, int m0) {
  // TMA-staged fine tiles: whole 32-column tiles per row, tiles no larger than the grid,
  // slices stored back to back (sfine = sf slabs), 16-byte aligned base
  if (gf.pitch % ITX == 0 && gc.n >= I3CW && gc.pitch % 4 == 0 && sfine == (long long)sf * gf.slab &&
      ((uintptr_t)Uf & 15) == 0 && ((uintptr_t)dU & 15) == 0 && tma::encoder() != nullptr)
    return order == 2 ? launch_interp_space3d_tma<T, 2>(L, gf, gc, sf, dU, Uf, batch, m0)
                      : launch_interp_space3d_tma<T, 4>(L, gf, gc, sf, dU, Uf, batch, m0);
  const int ntx = (gf.n + ITX - 1) / ITX, nty = (gf.n + ITY - 1) / ITY, ntz = (gf.n + ITZ - 1) / ITZ;
  dim3 gr(ntx, nty, ntz * batch);
  if (order == 2)
    interp_space3d_kernel<T, 2><<<gr, 256, 0, L.stream>>>(gf, gc, sf, (const T *)dU, Uf, sfine, ntz, m0);
  else
    interp_space3d_kernel<T, 4><<<gr, 256, 0, L.stream>>>(gf, gc, sf, (const T *)dU, Uf, sfine, ntz, m0);
  return cudaSuccess;
}

cudaError_t k_interp_space_add(const Launch &L, const Grid &gf, const Grid &gc, int order, int sf, Prec pr,
                               const void *dU, double *Uf, long long sfine, int batch, int m0) {
  Scope sc(L, K_INTERP, gf, batch * (sf - m0), pr);
  if (gf.dim == 3 && (long long)((gf.n + ITZ - 1) / ITZ) * batch <= 65535) {
    const cudaError_t e = pr == F64 ? launch_interp_space3d<double>(L, gf, gc, order, sf, dU, Uf, sfine, batch, m0)
                                    : launch_interp_space3d<float>(L, gf, gc, order, sf, dU, Uf, sfine, batch, m0);
    const cudaError_t e2 = sc.done();
    return e != cudaSuccess ? e : e2;
  }
  if (pr == F64)
    PMG_DIM_SWITCH(gf.dim, (launch_interp_space<D, double>(L, gf, gc, order, sf, dU, Uf, sfine, batch, m0)))
  else
    PMG_DIM_SWITCH(gf.dim, (launch_interp_space<D, float>(L, gf, gc, order, sf, dU, Uf, sfine, batch, m0)))
  return sc.done();
}

cudaError_t k_colloc_residual(const Launch &L, const Grid &g, const ResCoef &cf, const double *U, const double *F,
                              long long stride, int batch, unsigned long long *out) {
  dim3 gr, bl;
  config(g, batch, gr, bl);
  Scope sc(L, K_COLLOC, g, batch, 0);
  colloc_residual_kernel<<<gr, bl, 0, L.stream>>>(g, cf, U, F, stride, batch, out);
  return sc.done();
}

cudaError_t k_fine_rhs_residual(const Launch &L, const Grid &g, const ResCoef &cf, double nu, const double *U,
                                long long stride, double *q, long long sq, int batch, unsigned long long *res,
                                bool chained) {
  dim3 gr, bl;
  config(g, batch, gr, bl);
  Scope sc(L, K_FINE_RHS, g, batch, 0);
  ResCoef scaled = cf;
  for (int m = 0; m < cf.s; ++m)
    for (int jn = 0; jn < cf.s; ++jn) {
      scaled.dtQ[m][jn] = nu * g.ih2 * cf.dtQ[m][jn];
      if (m + 1 < cf.s) scaled.dS[m][jn] = nu * g.ih2 * cf.dS[m][jn];
    }
  const long long total = (long long)g.nz * g.ny * g.pitch;
  long long nblk = (total + 255) / 256;
  if (nblk > 152 * 8) nblk = 152 * 8;
  const size_t csmem = sizeof(unsigned long long) * batch;
  // (the chained variant serves the second-order stencil only)
  chained = chained && batch > 1 && csmem <= 48 * 1024 && g.order != 4;
#define PMG_FRR(S_)                                                                                            \
  case S_:                                                                                                     \
    if (chained)                                                                                               \
      PMG_DIM_SWITCH(g.dim, (fine_rhs_chain_kernel<D, S_><<<(unsigned)nblk, 256, csmem, L.stream>>>(           \
                                g, scaled, U, stride, q, sq, batch, res)))                                     \
    else if (g.order == 4)                                                                                     \
      PMG_DIM_SWITCH(g.dim, (fine_rhs_residual_kernel<D, S_, true><<<gr, bl, 0, L.stream>>>(                   \
                                g, scaled, U, stride, q, sq, batch, res)))                                     \
    else                                                                                                       \
      PMG_DIM_SWITCH(g.dim, (fine_rhs_residual_kernel<D, S_, false><<<gr, bl, 0, L.stream>>>(                  \
                                g, scaled, U, stride, q, sq, batch, res)));                                    \
    break;
  switch (cf.s) {
    PMG_FRR(2) PMG_FRR(3) PMG_FRR(4) PMG_FRR(5) PMG_FRR(6) PMG_FRR(7) PMG_FRR(8) PMG_FRR(9)
    default: break;
  }
#undef PMG_FRR
  return sc.done();
}

cudaError_t k_fas_restrict_u(const Launch &L, const Grid &gf, const Grid &gc, const FASCoef &cf, const double *Uf,
                             long long sfine, double *Uc, double *Fc, double *tau, double *Uc0, long long scoarse,
                             int batch) {
  dim3 gr, bl;
  config(gc, batch, gr, bl);
  Scope sc(L, K_FAS, gc, batch, 0);
  FASCoef cs = cf;  // fine weights times nu / h_f^2; rows with no quadrature weight flagged
  cs.zero_rows = 0;
  for (int j = 0; j < cf.sc; ++j) {
    bool zero = true;
    for (int i = 0; i < cf.sf; ++i) {
      zero = zero && cf.dtQf[j][i] == 0.0;
      cs.dtQf[j][i] = cf.nu * gf.ih2 * cf.dtQf[j][i];
    }
    for (int i = 0; i < cf.sc; ++i) zero = zero && cf.dtQc[j][i] == 0.0;
    if (zero) cs.zero_rows |= 1 << j;
  }
  // node counts as compile-time constants: coarse nodes are a subset of the fine ones
#define PMG_FAS(SF_, SC_)                                                                                        \
  if (cf.sf == SF_ && cf.sc == SC_) {                                                                            \
    PMG_DIM_SWITCH(gf.dim, (fas_restrict_u_kernel<D, SF_, SC_><<<gr, bl, 0, L.stream>>>(gf, gc, cs, Uf, sfine, Uc, Fc, \
                                                                                         tau, Uc0, scoarse, batch))); \
    return sc.done();                                                                                          \
  }
  PMG_FAS(5, 3) PMG_FAS(3, 2) PMG_FAS(5, 2) PMG_FAS(9, 3)
#undef PMG_FAS
  PMG_DIM_SWITCH(gf.dim, (fas_restrict_u_kernel<D, 0, 0><<<gr, bl, 0, L.stream>>>(gf, gc, cs, Uf, sfine, Uc, Fc, tau,
                                                                                    Uc0, scoarse, batch)))
  return sc.done();
}

cudaError_t k_widen_check(cudaStream_t st, unsigned long long *bad) {
  widen_check_kernel<<<152 * 16, 256, 0, st>>>(bad);
  return cudaGetLastError();
}

cudaError_t k_narrow_check(cudaStream_t st, long long count, unsigned long long seed, unsigned long long *bad) {
  narrow_check_kernel<<<152 * 8, 256, 0, st>>>(count, seed, bad);
  return cudaGetLastError();
}

cudaError_t k_copy(const Launch &L, const Grid &g, const double *src, long long ss, double *dst, long long sd,
                   int batch) {
  dim3 gr, bl;
  config(g, batch, gr, bl);
  Scope sc(L, K_COPY, g, batch, 0);
  if (flat_ok(g, batch, ss | sd)) {
    copy_flat_kernel<<<flat_grid(g.slab, batch), 256, 0, L.stream>>>(g.slab, g.pitch, src, ss, dst, sd);
    return sc.done();
  }
  copy_kernel<<<gr, bl, 0, L.stream>>>(g, src, ss, dst, sd, batch);
  return sc.done();
}

cudaError_t k_pack(const Launch &L, const Grid &g, const double *dense, long long sdense, double *pad, long long spad,
                   int batch) {
  dim3 gr, bl;
  config(g, batch, gr, bl);
  Scope sc(L, K_PACK, g, batch, 0);
  pack_kernel<<<gr, bl, 0, L.stream>>>(g, dense, sdense, pad, spad, batch);
  return sc.done();
}

cudaError_t k_unpack(const Launch &L, const Grid &g, const double *pad, long long spad, double *dense,
                     long long sdense, int batch) {
  dim3 gr, bl;
  config(g, batch, gr, bl);
  Scope sc(L, K_UNPACK, g, batch, 0);
  unpack_kernel<<<gr, bl, 0, L.stream>>>(g, pad, spad, dense, sdense, batch);
  return sc.done();
}

int interp_timeouts() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_interp_timeout, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_interp_timeout, &zero, sizeof(int));
  }
  return v;
}

}  // namespace pmg
