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

template <int DIM, typename T>
cudaError_t launch_tail(const Launch &L, const VTailDesc &d, const void *minv, const void *f, long long fslab,
                        int fpitch, const void *ein, void *e, long long eslab, int epitch, int batch) {
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
