// vcycle_coop.cu -- the V-cycles of one sub-step solve on a single grid (the serial
// coarse chain of PFASST) as one persistent, cooperatively launched kernel.
//
// A single 127^3 grid does not fill the GPU, and one V-cycle with red-black smoothing
// is about 30 launches of which most work on grids of 31^3 and smaller, so the coarse
// chain is bound by launch latency.  Here every CTA stays resident for the whole solve
// (cooperative launch: all CTAs co-resident, one per SM) and the phases of the V-cycles
// -- each colour of each smoothing sweep, the residual, its full weighting, the exact
// 3^d solve, the prolongation -- are separated by a grid-wide barrier instead of kernel
// boundaries.  The per-point arithmetic is that of the per-level kernels in kernels.cu
// (same formulas, same order of the sums), so the results are bitwise the same.  The
// residual of a level is formed once per fine point into a scratch array and weighted in
// a second phase: evaluated inside the weighting, as the per-level kernel does, each
// coarse point would chain 27 stencils of L2 loads on far too few warps to hide them.
//
// Grid barrier: one 32-bit counter in device memory, zeroed before the launch; barrier
// number b is passed once the counter reaches (b + 1) * gridDim.x.  Every wait is
// bounded (about 2 s of SM clock); a CTA that gives up sets a device flag and returns,
// the other CTAs then give up at their own next wait, and the host reports
// PMG_ERR_TIMEOUT.
#include <cstdio>

#include "pmg_internal.cuh"

namespace pmg {
namespace {

__device__ int g_coop_timeout;  // set by a timed-out grid barrier

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// grid-wide barrier number `b` (0, 1, 2, ... in program order); false on a timeout.
// bar.sync orders the CTA's writes before thread 0's release-add; thread 0's acquire
// loads and the closing bar.sync order every later read of the CTA after the other CTAs'
// writes
__device__ __forceinline__ bool grid_sync(unsigned *count, unsigned b) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    const unsigned target = (b + 1u) * gridDim.x;
    if (ld_acquire_u32(count) < target) {
      const long long t0 = clock64();
      while (ld_acquire_u32(count) < target) {
        if (clock64() - t0 > 4000000000LL) {  // ~2 s at 2 GHz
          ok = 0;
          break;
        }
      }
    }
  }
  return __syncthreads_and(ok) != 0;
}

// level data of the solve, finest first (index 0 = the solve's top level)
struct CoopLevel {
  int n, pitch;       // interior points per axis, row pitch (n + 1)
  long long slab;     // elements of one grid function
  double ih2;         // 1 / h^2 of the level
  void *e, *f, *r;    // correction, right-hand side, residual scratch
};

struct CoopArgs {
  CoopLevel lev[kMaxLevels];
  int L;              // levels in the solve (>= 2)
  double c, omega;
  int nu1, nu2, nv;   // V(nu1, nu2), nv cycles
  const void *minv;   // exact inverse on the coarsest (3^d) level
  double *u;          // u += e after the last cycle
  unsigned *count;    // barrier counter
};

// rows of a level are dealt to warps; x along the lanes
template <int DIM>
__device__ __forceinline__ void row_of(int r, int n, int &j, int &k) {
  if (DIM == 3) {
    k = r / n;
    j = r - k * n;
  } else {
    k = 0;
    j = r;
  }
}

// (no __restrict__ in this file: every array is written in some phase of the kernel and
// read by other CTAs after a grid barrier, so no load may take the read-only path)
template <int DIM, typename T>
__device__ __forceinline__ T nbsum_c(const T *u, int n, int pitch, int i, int j, int k, long long off) {
  T s = (i > 0 ? u[off - 1] : T(0)) + (i < n - 1 ? u[off + 1] : T(0));
  s += (j > 0 ? u[off - pitch] : T(0)) + (j < n - 1 ? u[off + pitch] : T(0));
  if (DIM >= 3) {
    const long long pl = (long long)n * pitch;
    s += (k > 0 ? u[off - pl] : T(0)) + (k < n - 1 ? u[off + pl] : T(0));
  }
  return s;
}

// linear interpolation taps of fine 0-based index i onto coarse 0-based indices
__device__ __forceinline__ int lin_taps_c(int i, int nc, int *idx, float *w) {
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

// threads per CTA: 768 in FP32 (as many as the registers allow without spills: more warps
// to cover the L2 latency of the stencil loads), 512 in FP64
template <typename T>
constexpr int coop_threads() { return sizeof(T) == 4 ? 768 : 512; }

// grids of at most this many points per axis run in CTA 0 alone, with block barriers
constexpr int kCoopLocalN = 15;

template <int DIM, typename T>
__global__ void __launch_bounds__(coop_threads<T>(), 1) vcycle_coop_kernel(CoopArgs A) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, gnwarps = (gridDim.x * blockDim.x) >> 5;
  const int lwarp = threadIdx.x >> 5, lnwarps = blockDim.x >> 5;
  unsigned nb = 0;  // grid barriers passed
  const T omega = (T)A.omega;
  // one red-black colour on level l over the points of that colour (first: the first
  // sweep from e = 0, which also clears the other colour); two points per lane in flight
  auto colour_pass = [&](int l, int colour, bool first, int warp, int nwarps) {
    const CoopLevel &v = A.lev[l];
    T *e = (T *)v.e;
    const T *f = (const T *)v.f;
    const T a = (T)A.c * (T)v.ih2, D = T(1) + T(2 * DIM) * a;  // as the per-level kernels form it
    const int rows = DIM == 3 ? v.n * v.n : v.n;
    for (int r = warp; r < rows; r += nwarps) {
      int j, k;
      row_of<DIM>(r, v.n, j, k);
      const long long ro = ((long long)k * v.n + j) * v.pitch;
      if (first && colour == 0) {
        for (int i = lane; i < v.n; i += 32) {
          const long long o = ro + i;
          e[o] = ((i + j + k + DIM) & 1) == 0 ? omega * (f[o] / D) : T(0);
        }
        continue;
      }
      const int i0 = (colour + j + k + DIM) & 1;  // first x of this colour in the row
      for (int i = i0 + 2 * lane; i < v.n; i += 128) {
        const int i2 = i + 64;
        const long long o = ro + i, o2 = ro + i2;
        const T g1 = (f[o] + a * nbsum_c<DIM>(e, v.n, v.pitch, i, j, k, o)) / D;
        T g2 = T(0), e2 = T(0);
        if (i2 < v.n) {
          g2 = (f[o2] + a * nbsum_c<DIM>(e, v.n, v.pitch, i2, j, k, o2)) / D;
          e2 = e[o2];
        }
        e[o] = (T(1) - omega) * e[o] + omega * g1;
        if (i2 < v.n) e[o2] = (T(1) - omega) * e2 + omega * g2;
      }
    }
  };
  // residual r = f - (I - c Lap) e on level l, into its scratch array (the same
  // expression as the per-level restriction kernel evaluates at every fine point)
  auto residual_pass = [&](int l, int warp, int nwarps) {
    const CoopLevel &vf = A.lev[l];
    const T a = (T)A.c * (T)vf.ih2;
    const T *e = (const T *)vf.e, *fp = (const T *)vf.f;
    T *rs = (T *)vf.r;
    const int rows = DIM == 3 ? vf.n * vf.n : vf.n;
    for (int r = warp; r < rows; r += nwarps) {
      int j, k;
      row_of<DIM>(r, vf.n, j, k);
      const long long ro = ((long long)k * vf.n + j) * vf.pitch;
      for (int i = lane; i < vf.n; i += 32) {
        const long long fo = ro + i;
        const T ec = e[fo];
        rs[fo] = fp[fo] - (ec - a * (nbsum_c<DIM>(e, vf.n, vf.pitch, i, j, k, fo) - T(2 * DIM) * ec));
      }
    }
  };
  // fc = full weighting of the residual of level l onto level l + 1
  auto weight_pass = [&](int l, int warp, int nwarps) {
    const CoopLevel &vf = A.lev[l], &vc = A.lev[l + 1];
    const T w3[3] = {T(0.25), T(0.5), T(0.25)};
    const T *rs = (const T *)vf.r;
    T *fc = (T *)vc.f;
    const int rows = DIM == 3 ? vc.n * vc.n : vc.n;
    for (int r = warp; r < rows; r += nwarps) {
      int j, k;
      row_of<DIM>(r, vc.n, j, k);
      for (int i = lane; i < vc.n; i += 32) {
        T acc = T(0);
#pragma unroll
        for (int cz = (DIM >= 3 ? -1 : 0); cz <= (DIM >= 3 ? 1 : 0); ++cz)
#pragma unroll
          for (int cy = -1; cy <= 1; ++cy)
#pragma unroll
            for (int cx = -1; cx <= 1; ++cx) {
              const int fi = 2 * i + 1 + cx, fj = 2 * j + 1 + cy, fk = DIM >= 3 ? 2 * k + 1 + cz : 0;
              T w = w3[cx + 1];
              w *= w3[cy + 1];
              if (DIM >= 3) w *= w3[cz + 1];
              acc += w * rs[((long long)fk * vf.n + fj) * vf.pitch + fi];
            }
        fc[((long long)k * vc.n + j) * vc.pitch + i] = acc;
      }
    }
  };
  // e_l += P e_{l+1} (d-linear)
  auto prolong_pass = [&](int l, int warp, int nwarps) {
    const CoopLevel &vf = A.lev[l], &vc = A.lev[l + 1];
    T *e = (T *)vf.e;
    const T *ec = (const T *)vc.e;
    const int rows = DIM == 3 ? vf.n * vf.n : vf.n;
    for (int r = warp; r < rows; r += nwarps) {
      int j, k;
      row_of<DIM>(r, vf.n, j, k);
      int iy[2], iz[2] = {0, 0};
      float wy[2], wz[2] = {1.f, 1.f};
      const int ty = lin_taps_c(j, vc.n, iy, wy);
      const int tz = DIM >= 3 ? lin_taps_c(k, vc.n, iz, wz) : 1;
      for (int i = lane; i < vf.n; i += 32) {
        int ix[2];
        float wx[2];
        const int tx = lin_taps_c(i, vc.n, ix, wx);
        T acc = T(0);
        for (int cz = 0; cz < tz; ++cz)
          for (int cy = 0; cy < ty; ++cy)
            for (int cx = 0; cx < tx; ++cx)
              acc += T(wx[cx] * wy[cy] * wz[cz]) * ec[((long long)iz[cz] * vc.n + iy[cy]) * vc.pitch + ix[cx]];
        e[((long long)k * vf.n + j) * vf.pitch + i] += acc;
      }
    }
  };
  // exact solve on the coarsest level: e = Minv f (threads of the given warps)
  auto coarse_pass = [&](int warp, int nwarps) {
    constexpr int N3 = DIM == 2 ? 9 : 27;
    const CoopLevel &v = A.lev[A.L - 1];
    const T *minv = (const T *)A.minv, *f = (const T *)v.f;
    T *e = (T *)v.e;
    const int t = warp * 32 + lane;
    if (t < N3) {
      const int p = t, pi = p % 3, pj = (p / 3) % 3, pk = p / 9;
      T acc = T(0);
      for (int q = 0; q < N3; ++q) {
        const int qi = q % 3, qj = (q / 3) % 3, qk = q / 9;
        acc += minv[p * N3 + q] * f[((long long)qk * v.n + qj) * v.pitch + qi];
      }
      e[((long long)pk * v.n + pj) * v.pitch + pi] = acc;
    }
  };
  // the first level that CTA 0 handles alone (its grid and every coarser one are small)
  int lb = A.L - 1;
  while (lb > 0 && A.lev[lb - 1].n <= kCoopLocalN) --lb;
  const bool cta0 = blockIdx.x == 0;
  bool ok = true;
  for (int cyc = 0; cyc < A.nv && ok; ++cyc) {
    // down, grid-wide, on the levels above lb
    for (int l = 0; l < lb && ok; ++l) {
      const bool zero = l > 0 || cyc == 0;
      for (int s = 0; s < A.nu1 && ok; ++s)
        for (int colour = 0; colour < 2 && ok; ++colour) {
          colour_pass(l, colour, zero && s == 0, gwarp, gnwarps);
          ok = grid_sync(A.count, nb++);
        }
      if (ok) {
        residual_pass(l, gwarp, gnwarps);
        ok = grid_sync(A.count, nb++);
      }
      if (ok) {
        weight_pass(l, gwarp, gnwarps);
        ok = grid_sync(A.count, nb++);
      }
    }
    // the bottom of the cycle from level lb, in CTA 0 with block barriers
    if (ok && cta0) {
      for (int l = lb; l + 1 < A.L; ++l) {
        const bool zero = l > 0 || cyc == 0;
        for (int s = 0; s < A.nu1; ++s)
          for (int colour = 0; colour < 2; ++colour) {
            colour_pass(l, colour, zero && s == 0, lwarp, lnwarps);
            __syncthreads();
          }
        residual_pass(l, lwarp, lnwarps);
        __syncthreads();
        weight_pass(l, lwarp, lnwarps);
        __syncthreads();
      }
      coarse_pass(lwarp, lnwarps);
      __syncthreads();
      for (int l = A.L - 2; l >= lb; --l) {
        prolong_pass(l, lwarp, lnwarps);
        __syncthreads();
        for (int s = 0; s < A.nu2; ++s)
          for (int colour = 0; colour < 2; ++colour) {
            colour_pass(l, colour, false, lwarp, lnwarps);
            __syncthreads();
          }
      }
    }
    if (ok) ok = grid_sync(A.count, nb++);
    // up, grid-wide, on the levels above lb
    for (int l = lb - 1; l >= 0 && ok; --l) {
      prolong_pass(l, gwarp, gnwarps);
      ok = grid_sync(A.count, nb++);
      for (int s = 0; s < A.nu2 && ok; ++s)
        for (int colour = 0; colour < 2 && ok; ++colour) {
          colour_pass(l, colour, false, gwarp, gnwarps);
          ok = grid_sync(A.count, nb++);
        }
    }
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(&g_coop_timeout, 1);
    return;
  }
  if (A.u) {  // u += e on the top level (FP64 iterate)
    const CoopLevel &v = A.lev[0];
    const T *e = (const T *)v.e;
    const int rows = DIM == 3 ? v.n * v.n : v.n;
    for (int r = gwarp; r < rows; r += gnwarps) {
      int j, k;
      row_of<DIM>(r, v.n, j, k);
      const long long ro = ((long long)k * v.n + j) * v.pitch;
      for (int i = lane; i < v.n; i += 32) A.u[ro + i] += to_f64(e[ro + i]);
    }
  }
}

template <int DIM, typename T>
int coop_blocks() {
  static int blocks = -1;
  if (blocks < 0) {
    int dev = 0, sms = 0, per = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, vcycle_coop_kernel<DIM, T>, coop_threads<T>(), 0) != cudaSuccess) {
      cudaGetLastError();
      blocks = 0;
    } else {
      blocks = (coop && per >= 1) ? sms : 0;  // one CTA per SM
    }
  }
  return blocks;
}

}  // namespace

bool vcycle_coop_supported(const Grid &g0, int levels, int smoother_rbgs, int nu1) {
  return smoother_rbgs && nu1 >= 1 && (g0.dim == 2 || g0.dim == 3) && g0.order != 4 && levels >= 2 &&
         levels <= kMaxLevels;
}

cudaError_t k_vcycle_coop(const Launch &L, const Grid *lev, int nlev, Prec pr, double c, double omega, int nu1,
                          int nu2, int nv, void *const *e, void *const *f, void *const *r, const void *minv,
                          double *u, unsigned *count) {
  CoopArgs A;
  A.L = nlev;
  A.c = c;
  A.omega = omega;
  A.nu1 = nu1;
  A.nu2 = nu2;
  A.nv = nv;
  A.minv = minv;
  A.u = u;
  A.count = count;
  for (int l = 0; l < nlev; ++l) {
    A.lev[l].n = lev[l].n;
    A.lev[l].pitch = lev[l].pitch;
    A.lev[l].slab = lev[l].slab;
    A.lev[l].ih2 = lev[l].ih2;
    A.lev[l].e = e[l];
    A.lev[l].f = f[l];
    A.lev[l].r = r[l];
  }
  Scope sc(L, K_VCOOP, lev[0], 1, pr);
  cudaError_t err = cudaMemsetAsync(count, 0, sizeof(unsigned), L.stream);
  if (err != cudaSuccess) return err;
  // cooperative launch (every CTA co-resident), recorded as a kernel node under capture
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeCooperative;
  attr.val.cooperative = 1;
  cfg.blockDim = dim3(pr == F32 ? coop_threads<float>() : coop_threads<double>());
  cfg.dynamicSmemBytes = 0;
  cfg.stream = L.stream;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int blocks = 0;
  if (lev[0].dim == 3) {
    blocks = pr == F32 ? coop_blocks<3, float>() : coop_blocks<3, double>();
    cfg.gridDim = dim3(blocks > 0 ? blocks : 1);
    if (blocks > 0)
      err = pr == F32 ? cudaLaunchKernelEx(&cfg, vcycle_coop_kernel<3, float>, A)
                      : cudaLaunchKernelEx(&cfg, vcycle_coop_kernel<3, double>, A);
  } else {
    blocks = pr == F32 ? coop_blocks<2, float>() : coop_blocks<2, double>();
    cfg.gridDim = dim3(blocks > 0 ? blocks : 1);
    if (blocks > 0)
      err = pr == F32 ? cudaLaunchKernelEx(&cfg, vcycle_coop_kernel<2, float>, A)
                      : cudaLaunchKernelEx(&cfg, vcycle_coop_kernel<2, double>, A);
  }
  if (blocks <= 0) return cudaErrorNotSupported;
  cudaError_t e2 = sc.done();
  return err != cudaSuccess ? err : e2;
}

int coop_timeouts() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_coop_timeout, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_coop_timeout, &zero, sizeof(int));
  }
  return v;
}

}  // namespace pmg
