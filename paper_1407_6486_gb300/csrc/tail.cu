// tail.cu -- the bottom of a multigrid V-cycle in one launch.
//
// The coarse levels of a V-cycle (Sec. 4.1.1: smoothing, full-weighting restriction
// of the residual, exact solve on 3^d points, linear prolongation) hold few points,
// and run as separate kernels each costs a launch latency far above its work.  Here
// one CTA per grid runs every level from `top` down to the 3^d level and back up in
// shared memory: it reads the right-hand side of the top level, starts from a zero
// correction, and writes the top level's correction -- exactly the operations the
// per-level kernels would do, in the same order.  The top level may instead start from
// a given correction (a V-cycle that continues the previous one).
#include "pmg_internal.cuh"

namespace pmg {
namespace {

// one modest CTA per grid: it finds an SM quickly even while large kernels of other
// streams occupy the GPU
constexpr int kVTailThreads = 256;

// neighbour sum of dense level storage (zero outside)
template <int DIM, typename T>
__device__ __forceinline__ T dnb(const T *u, int n, int i, int j, int k, int idx) {
  T s = (i > 0 ? u[idx - 1] : T(0)) + (i < n - 1 ? u[idx + 1] : T(0));
  if (DIM >= 2) s += (j > 0 ? u[idx - n] : T(0)) + (j < n - 1 ? u[idx + n] : T(0));
  if (DIM >= 3) s += (k > 0 ? u[idx - n * n] : T(0)) + (k < n - 1 ? u[idx + n * n] : T(0));
  return s;
}

template <int DIM>
__device__ __forceinline__ void split(int idx, int n, int &i, int &j, int &k) {
  i = idx % n;
  j = DIM >= 2 ? (idx / n) % n : 0;
  k = DIM >= 3 ? idx / (n * n) : 0;
}

__device__ __forceinline__ int lin_taps_t(int i, int nc, int *idx, float *w) {
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

// one smoothing sweep on a level in shared memory; returns the buffer holding the result
// (Jacobi ping-pongs between e and e2)
template <int DIM, typename T>
__device__ T *tail_smooth(const VTailDesc &d, int n, T a, T *e, T *e2, const T *f, bool first) {
  const int N = DIM == 1 ? n : (DIM == 2 ? n * n : n * n * n);
  const T D = T(1) + T(2 * DIM) * a;
  const T omega = (T)d.omega;
  if (d.smoother == 0) {  // weighted Jacobi
    const T wD = omega / D;
    for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
      if (first) {
        e2[idx] = wD * f[idx];
      } else {
        int i, j, k;
        split<DIM>(idx, n, i, j, k);
        const T ec = e[idx];
        const T Le = ec - a * (dnb<DIM>(e, n, i, j, k, idx) - T(2 * DIM) * ec);
        e2[idx] = ec + wD * (f[idx] - Le);
      }
    }
    __syncthreads();
    return e2;
  }
  for (int colour = 0; colour < 2; ++colour) {  // red = even 1-based index sum, first
    for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
      int i, j, k;
      split<DIM>(idx, n, i, j, k);
      const int par = (i + j + k + DIM) & 1;
      if (par != colour) {
        if (first && colour == 0) e[idx] = T(0);
        continue;
      }
      if (first && colour == 0) {
        e[idx] = omega * (f[idx] / D);
        continue;
      }
      const T gs = (f[idx] + a * dnb<DIM>(e, n, i, j, k, idx)) / D;
      e[idx] = (T(1) - omega) * e[idx] + omega * gs;
    }
    __syncthreads();
  }
  return e;
}

template <int DIM, typename T>
__global__ void __launch_bounds__(kVTailThreads) vtail_kernel(VTailDesc d, const T *__restrict__ minv,
                                                     const T *__restrict__ fin, long long fslab, int fpitch,
                                                     const T *ein, T *eout, long long eslab, int epitch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = (T *)smem_raw;
  // level arrays by offset (no local pointer tables)
  auto E = [&](int l) { return sm + d.off_e[l]; };
  auto E2 = [&](int l) { return sm + d.off_e2[l]; };
  auto F = [&](int l) { return sm + d.off_f[l]; };
  auto R = [&](int l) { return sm + d.off_r[l]; };
  const int b = blockIdx.x;
  auto npts = [&](int l) { return DIM == 1 ? d.n[l] : (DIM == 2 ? d.n[l] * d.n[l] : d.n[l] * d.n[l] * d.n[l]); };
  auto coef = [&](int l) { return (T)d.c * (T)((double)(d.n[l] + 1) * (double)(d.n[l] + 1)); };
  // right-hand side of the top level from the padded layout
  {
    const int n = d.n[0];
    for (int idx = threadIdx.x; idx < npts(0); idx += blockDim.x) {
      int i, j, k;
      split<DIM>(idx, n, i, j, k);
      F(0)[idx] = fin[b * fslab + ((long long)k * (DIM >= 2 ? n : 1) + j) * fpitch + i];
      if (ein) E(0)[idx] = ein[b * eslab + ((long long)k * (DIM >= 2 ? n : 1) + j) * epitch + i];
    }
  }
  __syncthreads();
  // down: pre-smoothing from zero, residual, full weighting
  for (int l = 0; l < d.nlev - 1; ++l) {
    const int n = d.n[l], N = npts(l);
    const T a = coef(l);
    T *cur = E(l);
    const bool zero = l > 0 || ein == nullptr;  // the top level may start from a given correction
    if (d.nu1 == 0 && zero) {
      for (int idx = threadIdx.x; idx < N; idx += blockDim.x) cur[idx] = T(0);
      __syncthreads();
    }
    for (int s = 0; s < d.nu1; ++s)
      cur = tail_smooth<DIM, T>(d, n, a, cur, cur == E(l) ? E2(l) : E(l), F(l), zero && s == 0);
    if (cur != E(l)) {  // keep the level's correction in E
      for (int idx = threadIdx.x; idx < N; idx += blockDim.x) E(l)[idx] = cur[idx];
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
      int i, j, k;
      split<DIM>(idx, n, i, j, k);
      const T ec = E(l)[idx];
      R(l)[idx] = F(l)[idx] - (ec - a * (dnb<DIM>(E(l), n, i, j, k, idx) - T(2 * DIM) * ec));
    }
    __syncthreads();
    const int nc = d.n[l + 1], Nc = npts(l + 1);
    const T w3[3] = {T(0.25), T(0.5), T(0.25)};
    for (int idx = threadIdx.x; idx < Nc; idx += blockDim.x) {
      int i, j, k;
      split<DIM>(idx, nc, i, j, k);
      T acc = T(0);
      for (int cz = (DIM >= 3 ? -1 : 0); cz <= (DIM >= 3 ? 1 : 0); ++cz)
        for (int cy = (DIM >= 2 ? -1 : 0); cy <= (DIM >= 2 ? 1 : 0); ++cy)
          for (int cx = -1; cx <= 1; ++cx) {
            const int fi = 2 * i + 1 + cx, fj = DIM >= 2 ? 2 * j + 1 + cy : 0, fk = DIM >= 3 ? 2 * k + 1 + cz : 0;
            T w = w3[cx + 1];
            if (DIM >= 2) w *= w3[cy + 1];
            if (DIM >= 3) w *= w3[cz + 1];
            acc += w * R(l)[(fk * (DIM >= 2 ? n : 1) + fj) * n + fi];
          }
      F(l + 1)[idx] = acc;
    }
    __syncthreads();
  }
  // exact solve on the 3^d level
  {
    constexpr int N3 = DIM == 1 ? 3 : (DIM == 2 ? 9 : 27);
    const int lc = d.nlev - 1;
    for (int p = threadIdx.x; p < N3; p += blockDim.x) {
      T acc = T(0);
      for (int q = 0; q < N3; ++q) acc += minv[p * N3 + q] * F(lc)[q];
      E(lc)[p] = acc;
    }
    __syncthreads();
  }
  // up: linear prolongation added, post-smoothing
  for (int l = d.nlev - 2; l >= 0; --l) {
    const int n = d.n[l], N = npts(l), nc = d.n[l + 1];
    for (int idx = threadIdx.x; idx < N; idx += blockDim.x) {
      int i, j, k;
      split<DIM>(idx, n, i, j, k);
      int ix[2], iy[2] = {0, 0}, iz[2] = {0, 0};
      float wx[2], wy[2] = {1.f, 1.f}, wz[2] = {1.f, 1.f};
      const int tx = lin_taps_t(i, nc, ix, wx);
      const int ty = DIM >= 2 ? lin_taps_t(j, nc, iy, wy) : 1;
      const int tz = DIM >= 3 ? lin_taps_t(k, nc, iz, wz) : 1;
      T acc = T(0);
      for (int cz = 0; cz < tz; ++cz)
        for (int cy = 0; cy < ty; ++cy)
          for (int cx = 0; cx < tx; ++cx)
            acc += T(wx[cx] * wy[cy] * wz[cz]) * E(l + 1)[(iz[cz] * (DIM >= 2 ? nc : 1) + iy[cy]) * nc + ix[cx]];
      E(l)[idx] += acc;
    }
    __syncthreads();
    T *cur = E(l);
    const T a = coef(l);
    for (int s = 0; s < d.nu2; ++s) cur = tail_smooth<DIM, T>(d, n, a, cur, cur == E(l) ? E2(l) : E(l), F(l), false);
    if (cur != E(l)) {
      for (int idx = threadIdx.x; idx < N; idx += blockDim.x) E(l)[idx] = cur[idx];
      __syncthreads();
    }
  }
  // correction of the top level to the padded layout
  {
    const int n = d.n[0];
    for (int idx = threadIdx.x; idx < npts(0); idx += blockDim.x) {
      int i, j, k;
      split<DIM>(idx, n, i, j, k);
      eout[b * eslab + ((long long)k * (DIM >= 2 ? n : 1) + j) * epitch + i] = E(0)[idx];
    }
  }
}

// The same V-cycle bottom for 3D red-black Gauss-Seidel with a top level of at most
// 15^3 points: 1024 threads as a 16 x 8 x 8 block, thread (tx, ty, tz) owning the points
// (tx, ty + 8 s, tz + 8 t) of a level -- four on 15^3, one on 7^3 -- so no index is
// divided; every level array is stored with a zero halo ((n + 2)^3 entries) so that the
// stencil needs no bounds test, and a colour pass visits only its own points.  The
// operations and their order per point are those of vtail_kernel.
constexpr int kVTail3Threads = 1024;

// linear-interpolation taps of fine index i as two fixed slots (slot 1 unused at an even
// 1-based index; a slot outside the coarse grid is marked off): the taps lin_taps_t lists,
// in the same order
struct Taps2 {
  int i[2];
  float w[2];
  bool ok[2];
};
__device__ __forceinline__ Taps2 taps2(int i, int nc) {
  Taps2 t;
  const int i1 = i + 1;
  if ((i1 & 1) == 0) {
    t.i[0] = i1 / 2 - 1;
    t.w[0] = 1.0f;
    t.ok[0] = true;
    t.i[1] = 0;
    t.w[1] = 0.f;
    t.ok[1] = false;
  } else {
    t.i[0] = (i1 - 1) / 2 - 1;
    t.i[1] = (i1 + 1) / 2 - 1;
    t.w[0] = t.w[1] = 0.5f;
    t.ok[0] = t.i[0] >= 0;
    t.ok[1] = t.i[1] < nc;
  }
  return t;
}

__host__ __device__ __forceinline__ int vt3_pad(int n) { return (n + 2) * (n + 2) * (n + 2); }

template <typename T>
__global__ void __launch_bounds__(kVTail3Threads) vtail3d_rb_kernel(VTailDesc d, const T *__restrict__ minv,
                                                                    const T *__restrict__ fin, long long fslab,
                                                                    int fpitch, const T *ein, T *eout,
                                                                    long long eslab, int epitch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sm = (T *)smem_raw;
  const int tid = threadIdx.x, tx = tid & 15, ty = (tid >> 4) & 7, tz = tid >> 7;
  const int b = blockIdx.x;
  // level arrays by the offsets of the padded layout (vtail3d_layout); the e arrays,
  // which hold every level's e together, start at 0: zero them (halos and the corrections
  // that start from zero); f and r are written before they are read
  for (int q = tid; q < d.off_f[0]; q += kVTail3Threads) sm[q] = T(0);
  auto E = [&](int l) { return sm + d.off_e[l]; };
  auto F = [&](int l) { return sm + d.off_f[l]; };
  auto R = [&](int l) { return sm + d.off_r[l]; };
  auto coef = [&](int l) { return (T)d.c * (T)((double)(d.n[l] + 1) * (double)(d.n[l] + 1)); };
  // padded index of interior point (i, j, k) of a level with n points per axis
  auto P = [](int n, int i, int j, int k) { return (i + 1) + (n + 2) * ((j + 1) + (n + 2) * (k + 1)); };
  // neighbour sum in the order of dnb: (x- + x+) + (y- + y+) + (z- + z+)
  auto nb6 = [](const T *u, int p, int s1, int s2) {
    T s = u[p - 1] + u[p + 1];
    s += u[p - s1] + u[p + s1];
    s += u[p - s2] + u[p + s2];
    return s;
  };
  // this thread's points of a level: (tx, ty + 8 s, tz + 8 t) inside n^3
#define VT3_FOR(n)                                    \
  for (int k = tz; k < (n); k += 8)                   \
    for (int j = ty; j < (n); j += 8)                 \
      if (tx < (n))
  const T omega = (T)d.omega;
  // one red-black sweep of level l (first: from a zero correction)
  auto sweep = [&](int l, bool first) {
    const int n = d.n[l], s1 = n + 2, s2 = (n + 2) * (n + 2);
    const T a = coef(l), D = T(1) + T(6) * a;
    T *e = E(l);
    const T *f = F(l);
    for (int colour = 0; colour < 2; ++colour) {  // red = even 1-based index sum, first
      VT3_FOR(n) {
        const int i = tx;
        if (((i + j + k + 3) & 1) != colour) continue;
        const int p = P(n, i, j, k);
        if (first && colour == 0) {
          e[p] = omega * (f[p] / D);  // black entries are already zero
          continue;
        }
        const T gs = (f[p] + a * nb6(e, p, s1, s2)) / D;
        e[p] = (T(1) - omega) * e[p] + omega * gs;
      }
      __syncthreads();
    }
  };
  __syncthreads();
  {  // right-hand side (and initial correction) of the top level from the padded layout
    const int n = d.n[0];
    VT3_FOR(n) {
      const long long g = ((long long)k * n + j) * fpitch + tx;
      F(0)[P(n, tx, j, k)] = fin[b * fslab + g];
      if (ein) E(0)[P(n, tx, j, k)] = ein[b * eslab + ((long long)k * n + j) * epitch + tx];
    }
  }
  __syncthreads();
  // down: pre-smoothing, residual, full weighting
  for (int l = 0; l < d.nlev - 1; ++l) {
    const int n = d.n[l], s1 = n + 2, s2 = (n + 2) * (n + 2);
    const T a = coef(l);
    const bool zero = l > 0 || ein == nullptr;
    for (int s = 0; s < d.nu1; ++s) sweep(l, zero && s == 0);
    VT3_FOR(n) {
      const int p = P(n, tx, j, k);
      const T ec = E(l)[p];
      R(l)[p] = F(l)[p] - (ec - a * (nb6(E(l), p, s1, s2) - T(6) * ec));
    }
    __syncthreads();
    const int nc = d.n[l + 1];
    VT3_FOR(nc) {
      // unrolled: the weights are exact constants (products of 1/4 and 1/2)
      const T *r0 = R(l) + P(n, 2 * tx + 1, 2 * j + 1, 2 * k + 1);
      T acc = T(0);
#pragma unroll
      for (int cz = -1; cz <= 1; ++cz)
#pragma unroll
        for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
          for (int cx = -1; cx <= 1; ++cx) {
            T w = cx == 0 ? T(0.5) : T(0.25);
            w *= cy == 0 ? T(0.5) : T(0.25);
            w *= cz == 0 ? T(0.5) : T(0.25);
            acc += w * r0[cx + s1 * (cy + s1 * cz)];
          }
      F(l + 1)[P(nc, tx, j, k)] = acc;
    }
    __syncthreads();
  }
  {  // exact solve on the 3^3 level (dense order i + 3 j + 9 k of the inverse)
    const int lc = d.nlev - 1;
    if (tid < 27) {
      T acc = T(0);
      for (int q = 0; q < 27; ++q) acc += minv[tid * 27 + q] * F(lc)[P(3, q % 3, (q / 3) % 3, q / 9)];
      E(lc)[P(3, tid % 3, (tid / 3) % 3, tid / 9)] = acc;
    }
    __syncthreads();
  }
  // up: linear prolongation added, post-smoothing
  for (int l = d.nlev - 2; l >= 0; --l) {
    const int n = d.n[l], nc = d.n[l + 1];
    VT3_FOR(n) {
      // the taps of lin_taps_t, in its order, as two fixed slots per axis
      const Taps2 X = taps2(tx, nc), Y = taps2(j, nc), Z = taps2(k, nc);
      T acc = T(0);
#pragma unroll
      for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy)
#pragma unroll
          for (int cx = 0; cx < 2; ++cx)
            if (Z.ok[cz] && Y.ok[cy] && X.ok[cx])
              acc += T(X.w[cx] * Y.w[cy] * Z.w[cz]) * E(l + 1)[P(nc, X.i[cx], Y.i[cy], Z.i[cz])];
      E(l)[P(n, tx, j, k)] += acc;
    }
    __syncthreads();
    for (int s = 0; s < d.nu2; ++s) sweep(l, false);
  }
  {  // correction of the top level to the padded layout
    const int n = d.n[0];
    VT3_FOR(n) eout[b * eslab + ((long long)k * n + j) * epitch + tx] = E(0)[P(n, tx, j, k)];
  }
#undef VT3_FOR
}

// the padded layout of vtail3d_rb_kernel in d's offsets: the e arrays of all levels
// first, then f and r of each level; returns the shared-memory bytes
size_t vtail3d_layout(VTailDesc &d, size_t tsize) {
  int t = 0;
  for (int l = 0; l < d.nlev; ++l) {
    d.off_e[l] = t;
    t += vt3_pad(d.n[l]);
  }
  for (int l = 0; l < d.nlev; ++l) {
    d.off_f[l] = t;
    t += vt3_pad(d.n[l]);
    d.off_r[l] = t;
    t += vt3_pad(d.n[l]);
  }
  return (size_t)t * tsize;
}

template <int DIM, typename T>
cudaError_t launch_tail(const Launch &L, const VTailDesc &d, const void *minv, const void *f, long long fslab,
                        int fpitch, const void *ein, void *e, long long eslab, int epitch, int batch) {
  VTailDesc d3 = d;
  if (DIM == 3 && d.smoother == 1 && d.n[0] <= 15 && d.n[d.nlev - 1] == 3 &&
      vtail3d_layout(d3, sizeof(T)) <= kVTailMaxSmem) {
    const size_t smem = vtail3d_layout(d3, sizeof(T));
    static bool attr3 = false;
    if (!attr3) {
      cudaError_t err = cudaFuncSetAttribute(vtail3d_rb_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kVTailMaxSmem);
      if (err != cudaSuccess) return err;
      attr3 = true;
    }
    vtail3d_rb_kernel<T><<<batch, kVTail3Threads, smem, L.stream>>>(d3, (const T *)minv, (const T *)f, fslab, fpitch,
                                                                      (const T *)ein, (T *)e, eslab, epitch);
    return cudaGetLastError();
  }
  const size_t smem = d.smem_elems * sizeof(T);
  if (smem > kVTailMaxSmem) return cudaErrorInvalidValue;
  static bool attr = false;  // once per instantiation, before any capture uses it
  if (!attr) {
    cudaError_t err = cudaFuncSetAttribute(vtail_kernel<DIM, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kVTailMaxSmem);
    if (err != cudaSuccess) return err;
    attr = true;
  }
  vtail_kernel<DIM, T><<<batch, kVTailThreads, smem, L.stream>>>(d, (const T *)minv, (const T *)f, fslab, fpitch,
                                                          (const T *)ein, (T *)e, eslab, epitch);
  return cudaSuccess;
}

}  // namespace

size_t vtail_plan(int dim, int n_top, int nlev, int smoother, size_t tsize, VTailDesc &d) {
  d.nlev = nlev;
  size_t off = 0;
  int n = n_top;
  for (int l = 0; l < nlev; ++l) {
    const size_t N = dim == 1 ? n : (dim == 2 ? (size_t)n * n : (size_t)n * n * n);
    const size_t Np = (N + 3) & ~(size_t)3;  // 16-byte alignment of every array (FP32)
    d.n[l] = n;
    d.off_e[l] = (int)off;
    off += Np;
    d.off_f[l] = (int)off;
    off += Np;
    d.off_r[l] = (int)off;
    off += Np;
    if (smoother == 0) {
      d.off_e2[l] = (int)off;
      off += Np;
    } else {
      d.off_e2[l] = d.off_r[l];  // unused by Gauss-Seidel
    }
    n = (n - 1) / 2;
  }
  d.smem_elems = off;
  return off * tsize;
}

cudaError_t k_vcycle_tail(const Launch &L, const Grid &g_top, const VTailDesc &d, Prec pr, const void *minv,
                          const void *f, const void *e_in, void *e, int batch) {
  Scope sc(L, K_VTAIL, g_top, batch, pr);
  cudaError_t err = cudaSuccess;
  const long long sl = g_top.slab;
  const int pt = g_top.pitch;
  switch (g_top.dim * 2 + (pr == F32 ? 1 : 0)) {
    case 2: err = launch_tail<1, double>(L, d, minv, f, sl, pt, e_in, e, sl, pt, batch); break;
    case 3: err = launch_tail<1, float>(L, d, minv, f, sl, pt, e_in, e, sl, pt, batch); break;
    case 4: err = launch_tail<2, double>(L, d, minv, f, sl, pt, e_in, e, sl, pt, batch); break;
    case 5: err = launch_tail<2, float>(L, d, minv, f, sl, pt, e_in, e, sl, pt, batch); break;
    case 6: err = launch_tail<3, double>(L, d, minv, f, sl, pt, e_in, e, sl, pt, batch); break;
    default: err = launch_tail<3, float>(L, d, minv, f, sl, pt, e_in, e, sl, pt, batch); break;
  }
  cudaError_t e2 = sc.done();
  return err != cudaSuccess ? err : e2;
}

}  // namespace pmg
