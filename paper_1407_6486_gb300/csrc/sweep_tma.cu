// sweep_tma.cu -- red-black Gauss-Seidel sweep of (I - c Lap_h) e = f on batched 3D
// grids with TMA-staged planes (FP32, rows of 128 or 256 elements).
//
// The same sweep as rbgs_rows3d_kernel in stencil3d.cu (one pass: the red half-sweep
// on plane k, then the black half-sweep on plane k-1, marching along z; out of place
// e_in -> e_out, from e = 0, or fused with u += e), but the planes are not fetched by
// the threads: one elected thread streams each z-plane tile of e_in (rows y0-2 ..
// y0+FTY+1) and of f (rows y0-1 .. y0+FTY) into a ring of shared-memory slots with
// cp.async.bulk.tensor, DEPTH planes ahead of the computation, completing on one
// mbarrier per slot.  The tensor-map box covers whole rows (x = 0, 16-byte aligned); rows and
// planes outside the grid arrive as zeros (the Dirichlet wall).  The threads only
// compute, which keeps their register count low and the loads deep.
// The red half-sweep writes its results into the e slot of its plane, in place: a red
// point reads only black neighbours (and its own value), so the red updates of one plane
// do not interfere, and the black half-sweep then finds the red values of planes k-2,
// k-1, k and the old black values in the same slots.  Without a separate red buffer the
// ring holds two planes in flight at two CTAs per SM.
// One CTA barrier per plane: a thread computes the red points of plane k on the rows of
// its own black half-sweep of plane k-1, and a black point reads red values of plane k
// only at its own (x, y), so the only values that cross threads within a plane step --
// the red values of plane k-1 and the slots refilled by TMA -- are ordered by the barrier
// that ends the previous plane.
//
// Every wait on an mbarrier is bounded (about 2 s of SM clock); on a timeout the
// kernel records the fact in a device flag, stops at the end of the current plane,
// waits (bounded again) for the loads it still has in flight and returns; the host
// turns the flag into PMG_ERR_TIMEOUT.  A load that has not landed after that second
// wait could still write into shared memory the CTA has released: the host then
// reports the timeout and the caller should treat the CUDA context as suspect.
#include "pmg_internal.cuh"
#include "tma.cuh"

namespace pmg {
namespace {

using namespace tma;

constexpr int TTY = 8;             // output rows per tile
constexpr int TEY = TTY + 4;       // e_in rows staged per plane (y0-2 .. y0+TTY+1)
constexpr int TMY = TTY + 2;       // red / f rows (y0-1 .. y0+TTY)
constexpr int DEPTH = 2;           // planes in flight ahead of the computation
constexpr int NE = 4 + DEPTH;      // e_in slots: planes k-2 .. k+1 in use, DEPTH more in flight
constexpr int NF = 2 + DEPTH;      // f slots: planes k-1, k in use, DEPTH more in flight
constexpr int TNT = 512;           // threads per CTA (two CTAs per SM: ~112 KB of ring each)
constexpr int TZC = 32;            // default z planes per CTA

__device__ int g_sweep_timeout;    // set by a timed-out mbarrier wait

template <int NX, bool ZERO, bool UPD>
__global__ void __launch_bounds__(TNT, 2) rbgs_tma_kernel(const __grid_constant__ CUtensorMap tme,
                                                          const __grid_constant__ CUtensorMap tmf, Grid g, float a,
                                                          float iD, float omega, float *__restrict__ eout,
                                                          double *__restrict__ u, long long su, int nzc, int zchunk) {
  constexpr int NP = NX / 2;          // x-pairs per row
  constexpr int RS = TNT / NP;        // rows per round of the CTA
  constexpr int PB = (TTY + RS - 1) / RS;
  constexpr uint32_t EB = TEY * NX * 4, FB = TMY * NX * 4;
  extern __shared__ __align__(1024) unsigned char sm[];
  float2(*E)[TEY][NP] = (float2(*)[TEY][NP])sm;                                   // [NE]
  float2(*Fs)[TMY][NP] = (float2(*)[TMY][NP])(sm + NE * EB);                       // [NF]
  uint64_t *bar = (uint64_t *)(sm + NE * EB + NF * FB);                            // [NE + NF]
  __shared__ int s_bad;
  const int n = g.n, tid = threadIdx.x, px = tid % NP, ry = tid / NP, lane = tid & 31;
  const int y0 = blockIdx.y * TTY;
  const int zc = blockIdx.z % nzc, b = blockIdx.z / nzc;
  const int z0 = zc * zchunk, z1 = min(z0 + zchunk, n);
  const long long plane = (long long)g.ny * g.pitch;
  const unsigned full = 0xffffffffu;
  // ring positions: e plane p in slot (p - z0 + 2) % NE, f plane p in slot (p - z0 + 1) % NF;
  // the j-th use of a slot completes phase j of its barrier
  auto eslot = [&](int p) { return (p - z0 + 2) % NE; };  // p >= z0 - 2
  auto fslot = [&](int p) { return (p - z0 + 1) % NF; };  // p >= z0 - 1
  auto issue_e = [&](int p) {
    const int s = eslot(p);
    mbar_expect_tx(&bar[s], EB);
    tma_load_4d(&E[s][0][0], &tme, 0, y0 - 2, p, b, &bar[s]);
  };
  auto issue_f = [&](int p) {
    const int s = fslot(p);
    mbar_expect_tx(&bar[NE + s], FB);
    tma_load_4d(&Fs[s][0][0], &tmf, 0, y0 - 1, p, b, &bar[NE + s]);
  };
  // ring slots above a given one, wrapped (d < N)
  auto eup = [](int sl, int d) { return sl + d >= NE ? sl + d - NE : sl + d; };
  auto edn = [](int sl, int d) { return sl - d < 0 ? sl - d + NE : sl - d; };
  auto fup = [](int sl, int d) { return sl + d >= NF ? sl + d - NF : sl + d; };
  auto fdn = [](int sl, int d) { return sl - d < 0 ? sl - d + NF : sl - d; };
  // x neighbours of the pair c in smem row `row` (lanes, or smem at a warp edge, or 0)
  auto xnb = [&](float2 c, const float2 *row, float &left, float &right) {
    const float l = __shfl_up_sync(full, c.y, 1), r = __shfl_down_sync(full, c.x, 1);
    left = lane != 0 ? l : (px > 0 ? row[px - 1].y : 0.f);
    right = lane != 31 ? r : (px < NP - 1 ? row[px + 1].x : 0.f);
  };

  if (tid == 0) {
    for (int i = 0; i < NE + NF; ++i) mbar_init(&bar[i]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    s_bad = 0;
    if (!ZERO)
      for (int p = z0 - 2; p <= min(z0 - 1 + DEPTH, z1 + 1); ++p) issue_e(p);
    for (int p = z0 - 1; p <= min(z0 - 2 + DEPTH, z1); ++p) issue_f(p);
  }
  __syncthreads();
  bool ok = true;
  if (!ZERO) ok = mbar_wait(&bar[0], 0) && mbar_wait(&bar[1], 0);  // planes z0-2, z0-1: slots 0, 1, phase 0
  double2 upre[PB];  // UPD: this thread's u pairs of plane k-1, loaded before the red phase
  int kstop = z1;    // plane at which a timed-out CTA stopped
  // ring positions kept incrementally (the same for every thread): the e slot of plane k+1
  // and the phase of its barrier, the f slot of plane k and its phase
  int s1 = 2, sfk = 0;
  uint32_t ph1 = 0, phf = 0;
  for (int k = z0 - 1; k <= z1; ++k) {
    if (tid == 0) {  // refill the slots the previous plane released
      if (!ZERO && k + 1 + DEPTH <= z1 + 1) {
        const int sl = eup(s1, DEPTH);
        mbar_expect_tx(&bar[sl], EB);
        tma_load_4d(&E[sl][0][0], &tme, 0, y0 - 2, k + 1 + DEPTH, b, &bar[sl]);
      }
      if (k + DEPTH <= z1) {
        const int sl = fup(sfk, DEPTH);
        mbar_expect_tx(&bar[NE + sl], FB);
        tma_load_4d(&Fs[sl][0][0], &tmf, 0, y0 - 1, k + DEPTH, b, &bar[NE + sl]);
      }
    }
    if (UPD && k - 1 >= z0 && k - 1 < z1) {
#pragma unroll
      for (int h = 0; h < PB; ++h) {
        const int r = ry + RS * h, y = y0 + r;
        if (r < TTY && y < n) upre[h] = *(const double2 *)(u + b * su + (k - 1) * plane + (long long)y * g.pitch + 2 * px);
      }
    }
    if (ok && !ZERO) ok = mbar_wait(&bar[s1], ph1);
    if (ok) ok = mbar_wait(&bar[NE + sfk], phf);
    if (!ok) s_bad = 1;
    {  // red half-sweep on plane k, rows y0-1 .. y0+TTY, into the e slot of plane k
      const int se = edn(s1, 1), sl = edn(s1, 2), sh = s1, sf = sfk;
      const bool kin = k >= 0 && k < n;
#pragma unroll
      for (int h = 0; h <= PB; ++h) {
        // a thread takes the rows of its black half-sweep (then the black half-sweep of
        // plane k-1 finds the red values of plane k it needs -- those of its own points --
        // without a CTA barrier); the halo rows y0-1 and y0+TTY go to the rows ry = 0, 1
        int r;
        if (h < PB) {
          if (ry + RS * h >= TTY) continue;  // uniform per warp (a warp lies in one row)
          r = ry + RS * h + 1;
        } else {
          if (ry >= 2) continue;
          r = ry == 0 ? 0 : TMY - 1;
        }
        const int y = y0 - 1 + r;
        const bool yin = kin && y >= 0 && y < n;
        const float2 fv = Fs[sf][r][px];
        const int ro = ((y + k) & 1) ? 0 : 1;  // red: x + y + k odd
        const int xr = 2 * px + ro;
        if (ZERO) {
          // from e = 0 the slot was never loaded: write the whole pair (black lane zero)
          float2 out = make_float2(0.f, 0.f);
          const float v = (yin && xr < n) ? omega * ((ro ? fv.y : fv.x) * iD) : 0.f;
          if (ro) out.y = v; else out.x = v;
          E[se][r + 1][px] = out;
        } else {
          // reads of black values only (neighbours and, through the pair, the other lane);
          // the store touches only this pair's red lane
          const float2 c = E[se][r + 1][px];
          float left, right;
          xnb(c, E[se][r + 1], left, right);
          if (yin && xr < n) {
            const float2 up = E[se][r][px], dn = E[se][r + 2][px], zl = E[sl][r + 1][px], zh = E[sh][r + 1][px];
            float nb, fr, old;
            if (ro == 0) {
              nb = left + c.y + up.x + dn.x + zl.x + zh.x;
              fr = fv.x;
              old = c.x;
            } else {
              nb = c.x + right + up.y + dn.y + zl.y + zh.y;
              fr = fv.y;
              old = c.y;
            }
            const float gs = (fr + a * nb) * iD;
            const float v = omega == 1.f ? gs : old + omega * (gs - old);
            if (ro) E[se][r + 1][px].y = v; else E[se][r + 1][px].x = v;
          }
        }
      }
    }
    // no barrier here: a black point of plane k-1 reads red values of plane k only at its
    // own (x, y) -- written above by this thread -- and red values of planes k-1, k-2 and
    // old black values, all settled before the barrier that ended the previous plane
    const int kb = k - 1;  // black half-sweep on plane k-1, rows y0 .. y0+TTY-1
    if (kb >= z0 && kb < z1) {
      const int s0 = edn(s1, 2), sl = edn(s1, 3), sh = edn(s1, 1), sf = fdn(sfk, 1);
#pragma unroll
      for (int h = 0; h < PB; ++h) {
        const int r = ry + RS * h;
        if (r >= TTY) break;
        const int y = y0 + r;
        const float2 c = E[s0][r + 2][px];  // red lane updated, black lane old
        float left, right;
        xnb(c, E[s0][r + 2], left, right);
        if (y >= n) continue;
        const float2 up = E[s0][r + 1][px], dn = E[s0][r + 3][px], zl = E[sl][r + 2][px], zh = E[sh][r + 2][px];
        const float2 fv = Fs[sf][r + 1][px];
        const int bo = ((y + kb) & 1) ? 1 : 0;  // black: x + y + kb even
        float2 out = c;
        const int xb = 2 * px + bo;
        if (xb < n) {
          float nb, fr, old;
          if (bo == 0) {
            nb = left + c.y + up.x + dn.x + zl.x + zh.x;
            fr = fv.x;
            old = ZERO ? 0.f : c.x;
          } else {
            nb = c.x + right + up.y + dn.y + zl.y + zh.y;
            fr = fv.y;
            old = ZERO ? 0.f : c.y;
          }
          const float gs = (fr + a * nb) * iD;
          const float v = omega == 1.f ? gs : old + omega * (gs - old);
          if (bo) out.y = v; else out.x = v;
        }
        const long long o = kb * plane + (long long)y * g.pitch + 2 * px;
        if (UPD) {
          double2 w = upre[h];
          w.x += widen_exact(out.x);
          w.y += widen_exact(out.y);
          *(double2 *)(u + b * su + o) = w;
        } else {
          *(float2 *)(eout + b * g.slab + o) = out;
        }
      }
    }
    __syncthreads();  // slots of plane k-1 may be refilled now
    if (s_bad) {      // uniform: read after the barrier
      kstop = k;
      break;
    }
    if (++s1 == NE) { s1 = 0; ph1 ^= 1u; }
    if (++sfk == NF) { sfk = 0; phf ^= 1u; }
  }
  if (s_bad && tid == 0) {
    atomicExch(&g_sweep_timeout, 1);
    // Before the CTA's shared memory is released, wait (bounded again) for every load
    // still in flight.  A slot is refilled only after its previous load was waited for,
    // so at most the last load issued into each slot can be outstanding: the planes
    // issued last, up to one per slot.
    if (!ZERO) {
      const int last = min(kstop + 1 + DEPTH, z1 + 1);
      for (int p = max(z0 - 2, last - NE + 1); p <= last; ++p) mbar_wait(&bar[eslot(p)], ((p - z0 + 2) / NE) & 1);
    }
    const int lastf = min(kstop + DEPTH, z1);
    for (int p = max(z0 - 1, lastf - NF + 1); p <= lastf; ++p) mbar_wait(&bar[NE + fslot(p)], ((p - z0 + 1) / NF) & 1);
  }
}

// The same sweep with four consecutive x points per thread (a float4 of a staged row):
// 2 * NX threads, eight rows per round.  The colour of a row is uniform over its warp
// (a warp lies in one row), so each half-sweep takes one of two branches for the whole
// warp: the two points of the colour in the quad (positions 0, 2 or 1, 3), one x
// neighbour from the adjacent lane's quad by a shuffle (or from shared memory at a warp
// edge), the other three from the quad itself; 128-bit shared loads and stores.  The red
// half-sweep stores the whole quad (its other colour unchanged) in place.  Per-point
// arithmetic, summation order and ring schedule are those of rbgs_tma_kernel, so the
// results are bitwise the same.
template <int NX, bool ZERO, bool UPD>
__global__ void __launch_bounds__(2 * NX, 2) rbgs_tma4_kernel(const __grid_constant__ CUtensorMap tme,
                                                              const __grid_constant__ CUtensorMap tmf, Grid g,
                                                              float a, float iD, float omega,
                                                              float *__restrict__ eout, double *__restrict__ u,
                                                              long long su, int nzc, int zchunk) {
  constexpr int NQ = NX / 4;          // quads per row
  constexpr int RS = 8;               // rows per round of the CTA
  constexpr int PB = (TTY + RS - 1) / RS;
  constexpr uint32_t EB = TEY * NX * 4, FB = TMY * NX * 4;
  extern __shared__ __align__(1024) unsigned char sm[];
  float4(*E)[TEY][NQ] = (float4(*)[TEY][NQ])sm;                                   // [NE]
  float4(*Fs)[TMY][NQ] = (float4(*)[TMY][NQ])(sm + NE * EB);                       // [NF]
  uint64_t *bar = (uint64_t *)(sm + NE * EB + NF * FB);                            // [NE + NF]
  __shared__ int s_bad;
  const int n = g.n, tid = threadIdx.x, qx = tid % NQ, ry = tid / NQ, lane = tid & 31;
  const int x0 = 4 * qx;
  const int y0 = blockIdx.y * TTY;
  const int zc = blockIdx.z % nzc, b = blockIdx.z / nzc;
  const int z0 = zc * zchunk, z1 = min(z0 + zchunk, n);
  const long long plane = (long long)g.ny * g.pitch;
  const unsigned full = 0xffffffffu;
  auto eslot = [&](int p) { return (p - z0 + 2) % NE; };  // p >= z0 - 2
  auto fslot = [&](int p) { return (p - z0 + 1) % NF; };  // p >= z0 - 1
  auto issue_e = [&](int p) {
    const int s = eslot(p);
    mbar_expect_tx(&bar[s], EB);
    tma_load_4d(&E[s][0][0], &tme, 0, y0 - 2, p, b, &bar[s]);
  };
  auto issue_f = [&](int p) {
    const int s = fslot(p);
    mbar_expect_tx(&bar[NE + s], FB);
    tma_load_4d(&Fs[s][0][0], &tmf, 0, y0 - 1, p, b, &bar[NE + s]);
  };
  auto eup = [](int sl, int d) { return sl + d >= NE ? sl + d - NE : sl + d; };
  auto edn = [](int sl, int d) { return sl - d < 0 ? sl - d + NE : sl - d; };
  auto fup = [](int sl, int d) { return sl + d >= NF ? sl + d - NF : sl + d; };
  auto fdn = [](int sl, int d) { return sl - d < 0 ? sl - d + NF : sl - d; };
  // x neighbours outside the quad: the previous quad's last value, the next quad's first
  auto leftq = [&](const float4 &c, const float4 *row) {
    const float l = __shfl_up_sync(full, c.w, 1);
    return lane != 0 ? l : (qx > 0 ? row[qx - 1].w : 0.f);
  };
  auto rightq = [&](const float4 &c, const float4 *row) {
    const float r = __shfl_down_sync(full, c.x, 1);
    return lane != 31 ? r : (qx < NQ - 1 ? row[qx + 1].x : 0.f);
  };
  // relaxed Gauss-Seidel value of one point from its neighbour sum, f and old value
  auto relax = [&](float nb, float fr, float old) {
    const float gs = (fr + a * nb) * iD;
    return omega == 1.f ? gs : old + omega * (gs - old);
  };

  if (tid == 0) {
    for (int i = 0; i < NE + NF; ++i) mbar_init(&bar[i]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    s_bad = 0;
    if (!ZERO)
      for (int p = z0 - 2; p <= min(z0 - 1 + DEPTH, z1 + 1); ++p) issue_e(p);
    for (int p = z0 - 1; p <= min(z0 - 2 + DEPTH, z1); ++p) issue_f(p);
  }
  __syncthreads();
  bool ok = true;
  if (!ZERO) ok = mbar_wait(&bar[0], 0) && mbar_wait(&bar[1], 0);
  double2 upre[PB][2];
  int kstop = z1;
  int s1 = 2, sfk = 0;
  uint32_t ph1 = 0, phf = 0;
  for (int k = z0 - 1; k <= z1; ++k) {
    if (tid == 0) {
      if (!ZERO && k + 1 + DEPTH <= z1 + 1) {
        const int sl = eup(s1, DEPTH);
        mbar_expect_tx(&bar[sl], EB);
        tma_load_4d(&E[sl][0][0], &tme, 0, y0 - 2, k + 1 + DEPTH, b, &bar[sl]);
      }
      if (k + DEPTH <= z1) {
        const int sl = fup(sfk, DEPTH);
        mbar_expect_tx(&bar[NE + sl], FB);
        tma_load_4d(&Fs[sl][0][0], &tmf, 0, y0 - 1, k + DEPTH, b, &bar[NE + sl]);
      }
    }
    if (UPD && k - 1 >= z0 && k - 1 < z1) {
#pragma unroll
      for (int h = 0; h < PB; ++h) {
        const int r = ry + RS * h, y = y0 + r;
        if (r < TTY && y < n) {
          const double2 *up = (const double2 *)(u + b * su + (k - 1) * plane + (long long)y * g.pitch + x0);
          upre[h][0] = up[0];
          upre[h][1] = up[1];
        }
      }
    }
    if (ok && !ZERO) ok = mbar_wait(&bar[s1], ph1);
    if (ok) ok = mbar_wait(&bar[NE + sfk], phf);
    if (!ok) s_bad = 1;
    {  // red half-sweep on plane k, rows y0-1 .. y0+TTY, into the e slot of plane k
      const int se = edn(s1, 1), sl = edn(s1, 2), sh = s1, sf = sfk;
      const bool kin = k >= 0 && k < n;
#pragma unroll
      for (int h = 0; h <= PB; ++h) {
        // the rows of the thread's black half-sweep, then the halo rows (as rbgs_tma_kernel)
        int r;
        if (h < PB) {
          if (ry + RS * h >= TTY) continue;  // uniform per warp
          r = ry + RS * h + 1;
        } else {
          if (ry >= 2) continue;
          r = ry == 0 ? 0 : TMY - 1;
        }
        const int y = y0 - 1 + r;
        const bool yin = kin && y >= 0 && y < n;
        const float4 fv = Fs[sf][r][qx];
        const bool ro = ((y + k) & 1) == 0;  // red at x + y + k odd: odd positions when y + k is even
        if (ZERO) {
          // from e = 0 the slot was never loaded: write the whole quad (black lanes zero)
          float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
          if (yin) {
            if (ro) {
              out.y = omega * (fv.y * iD);
              if (x0 + 3 < n) out.w = omega * (fv.w * iD);
            } else {
              out.x = omega * (fv.x * iD);
              out.z = omega * (fv.z * iD);
            }
          }
          E[se][r + 1][qx] = out;
        } else {
          float4 c = E[se][r + 1][qx];
          if (ro) {
            const float right = rightq(c, E[se][r + 1]);
            if (yin) {
              const float4 up = E[se][r][qx], dn = E[se][r + 2][qx], zl = E[sl][r + 1][qx], zh = E[sh][r + 1][qx];
              const float v1 = relax(c.x + c.z + up.y + dn.y + zl.y + zh.y, fv.y, c.y);
              if (x0 + 3 < n) c.w = relax(c.z + right + up.w + dn.w + zl.w + zh.w, fv.w, c.w);
              c.y = v1;
              E[se][r + 1][qx] = c;
            }
          } else {
            const float left = leftq(c, E[se][r + 1]);
            if (yin) {
              const float4 up = E[se][r][qx], dn = E[se][r + 2][qx], zl = E[sl][r + 1][qx], zh = E[sh][r + 1][qx];
              const float v0 = relax(left + c.y + up.x + dn.x + zl.x + zh.x, fv.x, c.x);
              c.z = relax(c.y + c.w + up.z + dn.z + zl.z + zh.z, fv.z, c.z);
              c.x = v0;
              E[se][r + 1][qx] = c;
            }
          }
        }
      }
    }
    // no barrier here (see rbgs_tma_kernel)
    const int kb = k - 1;  // black half-sweep on plane k-1, rows y0 .. y0+TTY-1
    if (kb >= z0 && kb < z1) {
      const int s0 = edn(s1, 2), sl = edn(s1, 3), sh = edn(s1, 1), sf = fdn(sfk, 1);
#pragma unroll
      for (int h = 0; h < PB; ++h) {
        const int r = ry + RS * h;
        if (r >= TTY) break;
        const int y = y0 + r;
        float4 c = E[s0][r + 2][qx];  // red lanes updated, black lanes old
        const bool bo = ((y + kb) & 1) != 0;  // black at x + y + kb even: odd positions when y + kb is odd
        if (bo) {
          const float right = rightq(c, E[s0][r + 2]);
          if (y >= n) continue;
          const float4 up = E[s0][r + 1][qx], dn = E[s0][r + 3][qx], zl = E[sl][r + 2][qx], zh = E[sh][r + 2][qx];
          const float4 fv = Fs[sf][r + 1][qx];
          const float v1 = relax(c.x + c.z + up.y + dn.y + zl.y + zh.y, fv.y, ZERO ? 0.f : c.y);
          if (x0 + 3 < n) c.w = relax(c.z + right + up.w + dn.w + zl.w + zh.w, fv.w, ZERO ? 0.f : c.w);
          c.y = v1;
        } else {
          const float left = leftq(c, E[s0][r + 2]);
          if (y >= n) continue;
          const float4 up = E[s0][r + 1][qx], dn = E[s0][r + 3][qx], zl = E[sl][r + 2][qx], zh = E[sh][r + 2][qx];
          const float4 fv = Fs[sf][r + 1][qx];
          const float v0 = relax(left + c.y + up.x + dn.x + zl.x + zh.x, fv.x, ZERO ? 0.f : c.x);
          c.z = relax(c.y + c.w + up.z + dn.z + zl.z + zh.z, fv.z, ZERO ? 0.f : c.z);
          c.x = v0;
        }
        const long long o = kb * plane + (long long)y * g.pitch + x0;
        if (UPD) {
          double2 w0 = upre[h][0], w1 = upre[h][1];
          w0.x += widen_exact(c.x);
          w0.y += widen_exact(c.y);
          w1.x += widen_exact(c.z);
          w1.y += widen_exact(c.w);
          double2 *uo = (double2 *)(u + b * su + o);
          uo[0] = w0;
          uo[1] = w1;
        } else {
          *(float4 *)(eout + b * g.slab + o) = c;
        }
      }
    }
    __syncthreads();  // slots of plane k-1 may be refilled now
    if (s_bad) {
      kstop = k;
      break;
    }
    if (++s1 == NE) { s1 = 0; ph1 ^= 1u; }
    if (++sfk == NF) { sfk = 0; phf ^= 1u; }
  }
  if (s_bad && tid == 0) {
    atomicExch(&g_sweep_timeout, 1);
    // wait (bounded) for the loads still in flight, as in rbgs_tma_kernel
    if (!ZERO) {
      const int last = min(kstop + 1 + DEPTH, z1 + 1);
      for (int p = max(z0 - 2, last - NE + 1); p <= last; ++p) mbar_wait(&bar[eslot(p)], ((p - z0 + 2) / NE) & 1);
    }
    const int lastf = min(kstop + DEPTH, z1);
    for (int p = max(z0 - 1, lastf - NF + 1); p <= lastf; ++p) mbar_wait(&bar[NE + fslot(p)], ((p - z0 + 1) / NF) & 1);
  }
}

// ---------------------------------------------------------------- residual + restriction
//
// fc = full weighting of r = f - (I - c Lap_h) e on batched 3D grids (FP32), with the
// e and f planes of a coarse tile streamed by TMA into a shared-memory ring, RD planes
// ahead.  Coarse tile RX x RY points, RZC coarse planes per CTA; the fine residual of
// one plane is formed in shared memory (double-buffered, so one barrier per fine plane
// suffices) and weighted in x and y; the z weights (1/4, 1/2, 1/4) accumulate in a
// register across the three fine planes of each coarse plane.  Boxes start at fine
// x = 2 I0 - 4 (a multiple of 4 floats: 16-byte aligned) and rows or planes outside
// the grid arrive as zeros.
constexpr int RX = 32, RY = 8, RZC = 16;
constexpr int RBX = 2 * RX + 8;    // staged columns: fine x 2I0-4 .. 2I0+67
constexpr int REY = 2 * RY + 3;    // e rows: fine y 2J0-1 .. 2J0+17
constexpr int RFY = 2 * RY + 1;    // f and residual rows: fine y 2J0 .. 2J0+16
constexpr int RRX = 2 * RX + 1;    // residual columns: fine x 2I0 .. 2I0+64
constexpr int RRS = RRX + 1;       // residual row stride
constexpr int RD = 2;              // planes in flight ahead of the computation
constexpr int RNE = 3 + RD, RNF = 1 + RD;
constexpr int RNT = RX * RY;       // 256 threads: one coarse point each
constexpr uint32_t REB = REY * RBX * 4, RFB = RFY * RBX * 4;
constexpr uint32_t RES = (REB + 127) / 128 * 128, RFS = (RFB + 127) / 128 * 128;  // 128-byte aligned slots
constexpr size_t RSMEM = RNE * RES + RNF * RFS + 2 * RFY * RRS * 4 + (RNE + RNF) * 8;

__global__ void __launch_bounds__(RNT, 4) resrestrict_tma_kernel(const __grid_constant__ CUtensorMap tme,
                                                                 const __grid_constant__ CUtensorMap tmf, Grid gf,
                                                                 Grid gc, float a, float *__restrict__ fc, int nzc) {
  extern __shared__ __align__(128) unsigned char sm[];
  float *Eb = (float *)sm;                                   // RNE slots of [REY][RBX]
  float *Fb = (float *)(sm + RNE * RES);                     // RNF slots of [RFY][RBX]
  float *Rb = (float *)(sm + RNE * RES + RNF * RFS);         // 2 x [RFY][RRS]
  uint64_t *bar = (uint64_t *)(sm + RNE * RES + RNF * RFS + 2 * RFY * RRS * 4);
  __shared__ int s_bad;
  const int tid = threadIdx.x, nc = gc.n;
  const int I0 = blockIdx.x * RX, J0 = blockIdx.y * RY;
  const int zc = blockIdx.z % nzc, b = blockIdx.z / nzc;
  const int K0 = zc * RZC, K1 = min(K0 + RZC, nc);
  const int zb = 2 * K0, ze = 2 * K1;  // fine planes 2K .. 2K+2 feed coarse plane K
  // e plane p (zb-1 .. ze+1) in slot (p - zb + 1) % RNE, f plane p (zb .. ze) in slot
  // (p - zb) % RNF; the j-th use of a slot completes phase j of its barrier
  auto eslot = [&](int p) { return (p - zb + 1) % RNE; };
  auto fslot = [&](int p) { return (p - zb) % RNF; };
  auto issue_e = [&](int p) {
    const int sl = eslot(p);
    mbar_expect_tx(&bar[sl], REB);
    tma_load_4d((char *)Eb + sl * RES, &tme, 2 * I0 - 4, 2 * J0 - 1, p, b, &bar[sl]);
  };
  auto issue_f = [&](int p) {
    const int sl = fslot(p);
    mbar_expect_tx(&bar[RNE + sl], RFB);
    tma_load_4d((char *)Fb + sl * RFS, &tmf, 2 * I0 - 4, 2 * J0, p, b, &bar[RNE + sl]);
  };
  if (tid == 0) {
    for (int i = 0; i < RNE + RNF; ++i) mbar_init(&bar[i]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    s_bad = 0;
    for (int p = zb - 1; p <= min(zb + RD, ze + 1); ++p) issue_e(p);
    for (int p = zb; p <= min(zb + RD - 1, ze); ++p) issue_f(p);
  }
  __syncthreads();
  const int cx = tid % RX, cy = tid / RX;
  const int I = I0 + cx, J = J0 + cy;
  const long long cplane = (long long)gc.ny * gc.pitch;
  float acc = 0.f;
  // the residual points of a fine plane this thread forms: the same for every plane, so
  // their staged-tile offsets are computed once (eo: e and f tiles, ro: residual tile)
  constexpr int NQ = (RFY * RRX + RNT - 1) / RNT;
  int eo_q[NQ], ro_q[NQ];
#pragma unroll
  for (int i = 0; i < NQ; ++i) {
    const int q = tid + i * RNT, ry = q / RRX, rx = q % RRX;
    eo_q[i] = q < RFY * RRX ? (ry + 1) * RBX + rx + 4 : -1;
    ro_q[i] = ry * RRS + rx;
  }
  bool ok = mbar_wait(&bar[0], 0) && mbar_wait(&bar[1], 0);  // e planes zb-1, zb: slots 0, 1, phase 0
  int zstop = ze;  // plane at which a timed-out CTA stopped
  // ring positions kept incrementally: e slot of plane z+1 and its phase, f slot of plane z
  int s1 = 2, sfz = 0;
  uint32_t ph1 = 0, phf = 0;
  for (int z = zb; z <= ze; ++z) {
    const int s0 = s1 == 0 ? RNE - 1 : s1 - 1, sm1 = s0 == 0 ? RNE - 1 : s0 - 1;
    if (tid == 0) {  // refill the slots of planes z-2 (e) and z-1 (f), read before the last barrier
      if (z + 1 + RD <= ze + 1) {
        const int sl = s1 + RD >= RNE ? s1 + RD - RNE : s1 + RD;
        mbar_expect_tx(&bar[sl], REB);
        tma_load_4d((char *)Eb + sl * RES, &tme, 2 * I0 - 4, 2 * J0 - 1, z + 1 + RD, b, &bar[sl]);
      }
      if (z + RD <= ze) {
        const int sl = sfz + RD >= RNF ? sfz + RD - RNF : sfz + RD;
        mbar_expect_tx(&bar[RNE + sl], RFB);
        tma_load_4d((char *)Fb + sl * RFS, &tmf, 2 * I0 - 4, 2 * J0, z + RD, b, &bar[RNE + sl]);
      }
    }
    if (ok) ok = mbar_wait(&bar[s1], ph1);
    if (ok) ok = mbar_wait(&bar[RNE + sfz], phf);
    if (!ok) s_bad = 1;
    const float *E0 = Eb + s0 * (RES / 4), *El = Eb + sm1 * (RES / 4), *Eh = Eb + s1 * (RES / 4),
                *F0 = Fb + sfz * (RFS / 4);
    float *R = Rb + (z & 1) * RFY * RRS;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {  // residual of fine plane z
      const int eo = eo_q[i];
      if (eo < 0) break;
      const float ec = E0[eo];
      const float nb = E0[eo - 1] + E0[eo + 1] + E0[eo - RBX] + E0[eo + RBX] + El[eo] + Eh[eo];
      R[ro_q[i]] = F0[eo - RBX] - (ec - a * (nb - 6.f * ec));
    }
    if (++s1 == RNE) { s1 = 0; ph1 ^= 1u; }
    if (++sfz == RNF) { sfz = 0; phf ^= 1u; }
    __syncthreads();
    if (s_bad) {  // uniform: read after the barrier
      zstop = z;
      break;
    }
    // x-y full weighting at the thread's coarse point: fine x = 2I+1 is residual column
    // 2cx+1, fine y = 2J+1 is residual row 2cy+1
    const int c0 = 2 * cx + 1, r0 = 2 * cy + 1;
    const float *Rm = R + (r0 - 1) * RRS + c0, *Rc = R + r0 * RRS + c0, *Rp = R + (r0 + 1) * RRS + c0;
    const float rxy = 0.25f * (0.25f * Rm[-1] + 0.5f * Rm[0] + 0.25f * Rm[1]) +
                      0.5f * (0.25f * Rc[-1] + 0.5f * Rc[0] + 0.25f * Rc[1]) +
                      0.25f * (0.25f * Rp[-1] + 0.5f * Rp[0] + 0.25f * Rp[1]);
    if ((z & 1) == 0) {
      if (z > zb && I < nc && J < nc) fc[b * gc.slab + (z / 2 - 1) * cplane + (long long)J * gc.pitch + I] = acc + 0.25f * rxy;
      acc = 0.25f * rxy;
    } else {
      acc += 0.5f * rxy;
    }
  }
  if (s_bad && tid == 0) {
    atomicExch(&g_sweep_timeout, 1);
    // wait (bounded) for the last load issued into every slot, as in the sweep above
    const int laste = min(zstop + 1 + RD, ze + 1), lastf = min(zstop + RD, ze);
    for (int p = max(zb - 1, laste - RNE + 1); p <= laste; ++p) mbar_wait(&bar[eslot(p)], ((p - zb + 1) / RNE) & 1);
    for (int p = max(zb, lastf - RNF + 1); p <= lastf; ++p) mbar_wait(&bar[RNE + fslot(p)], ((p - zb) / RNF) & 1);
  }
}

// tensor map of a batch of padded grid functions: dims (pitch, n, n, batch), box of
// `rows` whole rows of one plane
bool make_map(CUtensorMap *m, const void *base, const Grid &g, int batch, int rows) {
  auto enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)g.pitch, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)batch};
  const cuuint64_t strides[3] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.ny * g.pitch * 4, (cuuint64_t)g.slab * 4};
  const cuuint32_t box[4] = {(cuuint32_t)g.pitch, (cuuint32_t)rows, 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tensor map with a box of box_x columns and `rows` rows of one plane
bool make_map_box(CUtensorMap *m, const void *base, const Grid &g, int batch, int box_x, int rows) {
  auto enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)g.pitch, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)batch};
  const cuuint64_t strides[3] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.ny * g.pitch * 4, (cuuint64_t)g.slab * 4};
  const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)rows, 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NX, bool ZERO, bool UPD>
cudaError_t launch_tma(const Launch &L, const Grid &g, float a, float iD, float omega, const void *ein, void *eout,
                       const void *f, double *u, long long su, int batch, int zchunk) {
  constexpr uint32_t EB = TEY * NX * 4, FB = TMY * NX * 4;
  const size_t smem = NE * EB + NF * FB + (NE + NF) * 8;
  static bool attr = false;
  if (!attr) {
    // two CTAs of ~112 KB per SM: ask for the largest shared-memory carveout
    cudaError_t e = cudaFuncSetAttribute(rbgs_tma_kernel<NX, ZERO, UPD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(rbgs_tma_kernel<NX, ZERO, UPD>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  CUtensorMap me, mf;
  if (!make_map(&mf, f, g, batch, TMY)) return cudaErrorInvalidValue;
  if (!make_map(&me, ZERO ? f : ein, g, batch, TEY)) return cudaErrorInvalidValue;  // unused when ZERO
  if (zchunk <= 0) zchunk = TZC;
  const int nty = (g.n + TTY - 1) / TTY, nzc = (g.n + zchunk - 1) / zchunk;
  dim3 gr(1, nty, nzc * batch);
  rbgs_tma_kernel<NX, ZERO, UPD><<<gr, TNT, smem, L.stream>>>(me, mf, g, a, iD, omega, (float *)eout, u, su, nzc,
                                                               zchunk);
  return cudaGetLastError();
}

template <int NX, bool ZERO, bool UPD>
cudaError_t launch_tma4(const Launch &L, const Grid &g, float a, float iD, float omega, const void *ein, void *eout,
                        const void *f, double *u, long long su, int batch, int zchunk) {
  constexpr uint32_t EB = TEY * NX * 4, FB = TMY * NX * 4;
  const size_t smem = NE * EB + NF * FB + (NE + NF) * 8;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(rbgs_tma4_kernel<NX, ZERO, UPD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(rbgs_tma4_kernel<NX, ZERO, UPD>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  CUtensorMap me, mf;
  if (!make_map(&mf, f, g, batch, TMY)) return cudaErrorInvalidValue;
  if (!make_map(&me, ZERO ? f : ein, g, batch, TEY)) return cudaErrorInvalidValue;  // unused when ZERO
  if (zchunk <= 0) zchunk = TZC;
  const int nty = (g.n + TTY - 1) / TTY, nzc = (g.n + zchunk - 1) / zchunk;
  dim3 gr(1, nty, nzc * batch);
  rbgs_tma4_kernel<NX, ZERO, UPD><<<gr, 2 * NX, smem, L.stream>>>(me, mf, g, a, iD, omega, (float *)eout, u, su,
                                                                   nzc, zchunk);
  return cudaGetLastError();
}

template <bool ZERO, bool UPD>
cudaError_t launch_tma_pitch(const Launch &L, const Grid &g, float a, float iD, float omega, const void *ein,
                             void *eout, const void *f, double *u, long long su, int batch, int zchunk) {
  if (g.pitch == 256) return launch_tma<256, ZERO, UPD>(L, g, a, iD, omega, ein, eout, f, u, su, batch, zchunk);
  return launch_tma<128, ZERO, UPD>(L, g, a, iD, omega, ein, eout, f, u, su, batch, zchunk);
}

template <bool ZERO, bool UPD>
cudaError_t launch_tma4_pitch(const Launch &L, const Grid &g, float a, float iD, float omega, const void *ein,
                              void *eout, const void *f, double *u, long long su, int batch, int zchunk) {
  if (g.pitch == 256) return launch_tma4<256, ZERO, UPD>(L, g, a, iD, omega, ein, eout, f, u, su, batch, zchunk);
  return launch_tma4<128, ZERO, UPD>(L, g, a, iD, omega, ein, eout, f, u, su, batch, zchunk);
}

}  // namespace

int rbgs_tma_threads(const Grid &g, bool quad) { return quad ? 2 * g.pitch : TNT; }

bool rbgs_tma_supported(const Grid &g, Prec pr) {
  return pr == F32 && g.dim == 3 && g.order != 4 && (g.pitch == 128 || g.pitch == 256) && encoder() != nullptr;
}

cudaError_t k_rbgs_sweep3d_tma(const Launch &L, const Grid &g, double c, double omega, const void *ein, void *eout,
                               const void *f, double *u, long long su, int batch, bool zero, bool update_u,
                               int zchunk, bool quad) {
  Scope sc(L, zero ? K_RBGS3D_ZERO : (update_u ? K_RBGS3D_UPD : K_RBGS3D), g, batch, F32);
  const float a = (float)(c * g.ih2), D = 1.f + 6.f * a, iD = 1.f / D, w = (float)omega;
  cudaError_t e;
  if (quad) {
    if (zero && update_u) e = launch_tma4_pitch<true, true>(L, g, a, iD, w, ein, eout, f, u, su, batch, zchunk);
    else if (zero) e = launch_tma4_pitch<true, false>(L, g, a, iD, w, ein, eout, f, u, su, batch, zchunk);
    else if (update_u) e = launch_tma4_pitch<false, true>(L, g, a, iD, w, ein, eout, f, u, su, batch, zchunk);
    else e = launch_tma4_pitch<false, false>(L, g, a, iD, w, ein, eout, f, u, su, batch, zchunk);
  } else if (zero && update_u) e = launch_tma_pitch<true, true>(L, g, a, iD, w, ein, eout, f, u, su, batch, zchunk);
  else if (zero) e = launch_tma_pitch<true, false>(L, g, a, iD, w, ein, eout, f, u, su, batch, zchunk);
  else if (update_u) e = launch_tma_pitch<false, true>(L, g, a, iD, w, ein, eout, f, u, su, batch, zchunk);
  else e = launch_tma_pitch<false, false>(L, g, a, iD, w, ein, eout, f, u, su, batch, zchunk);
  cudaError_t e2 = sc.done();
  return e != cudaSuccess ? e : e2;
}

bool resrestrict_tma_supported(const Grid &gf, Prec pr) {
  return pr == F32 && gf.dim == 3 && gf.order != 4 && gf.pitch >= 128 && encoder() != nullptr;
}

cudaError_t k_resrestrict3d_tma(const Launch &L, const Grid &gf, const Grid &gc, double c, const void *e, const void *f,
                                void *fc, int batch) {
  Scope sc(L, K_RESRESTRICT3D, gc, batch, F32);
  static bool attr = false;
  if (!attr) {
    cudaError_t er = cudaFuncSetAttribute(resrestrict_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)RSMEM);
    if (er != cudaSuccess) return er;
    attr = true;
  }
  CUtensorMap me, mf;
  if (!make_map_box(&me, e, gf, batch, RBX, REY) || !make_map_box(&mf, f, gf, batch, RBX, RFY))
    return cudaErrorInvalidValue;
  const int ntx = (gc.n + RX - 1) / RX, nty = (gc.n + RY - 1) / RY, nzc = (gc.n + RZC - 1) / RZC;
  dim3 gr(ntx, nty, nzc * batch);
  resrestrict_tma_kernel<<<gr, RNT, RSMEM, L.stream>>>(me, mf, gf, gc, (float)(c * gf.ih2), (float *)fc, nzc);
  cudaError_t er = cudaGetLastError();
  cudaError_t e2 = sc.done();
  return er != cudaSuccess ? er : e2;
}

int sweep_timeouts() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_sweep_timeout, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_sweep_timeout, &zero, sizeof(int));
  }
  return v;
}

}  // namespace pmg
