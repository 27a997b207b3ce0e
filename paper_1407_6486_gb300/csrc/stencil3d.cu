// stencil3d.cu -- tiled 3D multigrid kernels for the large grids (sm_103a).
//
// The generic kernels of kernels.cu touch every point with one thread and read
// the neighbours through the caches.  For large batched 3D grids these kernels
// instead stage x-y tiles of consecutive z planes in shared memory and march
// along z, so each grid function is read once from HBM per pass:
//   - rbgs_sweep3d: one full red-black Gauss-Seidel sweep (Sec. 4.1.2 smoother,
//     red = (i+j+k) even in 1-based indices) fused into a single pass: the red
//     half-sweep runs one plane ahead of the black one (a wavefront), on the tile
//     plus a one-point ring so the black points at the tile edge see updated red
//     neighbours.  Out of place (e_in -> e_out), optionally from e_in = 0, and
//     optionally fused with the final refinement update u += e (no e_out written).
//   - resrestrict3d: residual r = f - (I - c Lap_h) e and full weighting
//     (1/4, 1/2, 1/4)^3 in one pass; r is formed once per fine point in shared
//     memory, restricted in x and y there and accumulated over z in registers.
//   - prolong3d: e += P e_c with trilinear interpolation, one thread per coarse
//     cell updating its 2x2x2 fine points.
#include <type_traits>

#include "pmg_internal.cuh"

namespace pmg {
namespace {

constexpr int RTX = 64, RTY = 8, RZC = 32;      // sweep: output tile and default z chunk
constexpr int SX = RTX + 4;                     // smem row: column c <-> x = x0 - 2 + c
constexpr int EY = RTY + 4, MY = RTY + 2;       // e_in rows (two-point ring), red/f rows (one-point ring)

// Thread (tx, ty), 32 x 8, owns the x-pair (x0 + 2tx, x0 + 2tx + 1): each pair holds
// exactly one red and one black point, so neither half-sweep diverges.
template <typename T, bool ZERO, bool UPD>
__global__ void __launch_bounds__(256, 4) rbgs_sweep3d_kernel(Grid g, T a, T D, T omega, const T *__restrict__ ein,
                                                              T *__restrict__ eout, const T *__restrict__ f,
                                                              double *__restrict__ u, long long su, int nzc,
                                                              int zchunk) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T(*E)[EY][SX] = (T(*)[EY][SX])sm_raw;                      // [4][EY][SX]
  T(*M)[MY][SX] = (T(*)[MY][SX])(sm_raw + sizeof(T) * 4 * EY * SX);   // [3][MY][SX]
  T(*Fs)[MY][SX] = (T(*)[MY][SX])(sm_raw + sizeof(T) * (4 * EY + 3 * MY) * SX);  // [3][MY][SX]
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  const int n = g.n, tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int x0 = blockIdx.x * RTX, y0 = blockIdx.y * RTY;
  const int zc = blockIdx.z % nzc, b = blockIdx.z / nzc;
  const int z0 = zc * zchunk, z1 = min(z0 + zchunk, n);
  const long long plane = (long long)g.ny * g.pitch;
  const T *Eb = ein + b * g.slab;
  const T *Fb = f + b * g.slab;
  const int xi = x0 + 2 * tx;  // first x of this thread's pair
  // halo assignments: e ring columns {0,1,66,67} x 12 rows; f ring columns {1,66} x 10 rows
  const int eh_row = tid >> 2, eh_col = (tid & 3) < 2 ? (tid & 3) : SX - 4 + (tid & 3);
  const int fh_row = (tid - 64) >> 1, fh_col = (tid & 1) ? SX - 2 : 1;
  const bool has_eh = tid < 4 * EY, has_fh = tid >= 64 && tid < 64 + 2 * MY;

  T2 pe[2], pf[2];
  T pe_h = T(0), pf_h = T(0);
  auto fetch_pair = [&](const T *base, int k, int j) -> T2 {
    T2 v;
    v.x = T(0);
    v.y = T(0);
    if (k >= 0 && k < n && j >= 0 && j < n && xi < n) v = *(const T2 *)(base + k * plane + (long long)j * g.pitch + xi);
    return v;
  };
  auto fetch_one = [&](const T *base, int k, int j, int i) -> T {
    return (k >= 0 && k < n && j >= 0 && j < n && i >= 0 && i < n) ? base[k * plane + (long long)j * g.pitch + i] : T(0);
  };
  auto fetch_e = [&](int k) {
    pe[0] = fetch_pair(Eb, k, y0 - 2 + ty);
    if (ty < EY - 8) pe[1] = fetch_pair(Eb, k, y0 + 6 + ty);
    if (has_eh) pe_h = fetch_one(Eb, k, y0 - 2 + eh_row, x0 - 2 + eh_col);
  };
  auto store_e = [&](int k) {
    T(*S)[SX] = E[(k + 4) & 3];
    *(T2 *)&S[ty][2 + 2 * tx] = pe[0];
    if (ty < EY - 8) *(T2 *)&S[ty + 8][2 + 2 * tx] = pe[1];
    if (has_eh) S[eh_row][eh_col] = pe_h;
  };
  auto fetch_f = [&](int k) {
    pf[0] = fetch_pair(Fb, k, y0 - 1 + ty);
    if (ty < MY - 8) pf[1] = fetch_pair(Fb, k, y0 + 7 + ty);
    if (has_fh) pf_h = fetch_one(Fb, k, y0 - 1 + fh_row, x0 - 2 + fh_col);
  };
  auto store_f = [&](int k) {
    T(*S)[SX] = Fs[(k + 3) % 3];
    *(T2 *)&S[ty][2 + 2 * tx] = pf[0];
    if (ty < MY - 8) *(T2 *)&S[ty + 8][2 + 2 * tx] = pf[1];
    if (has_fh) S[fh_row][fh_col] = pf_h;
  };
  // red update (or copy of the black value) at smem row r (global y = y0 - 1 + r), column c
  auto red_at = [&](int k, int r, int c, int se, int sl, int sh, int sf) -> T {
    const int i = x0 - 2 + c, j = y0 - 1 + r;
    if (k < 0 || k >= n || i < 0 || i >= n || j < 0 || j >= n) return T(0);
    const T old = ZERO ? T(0) : E[se][r + 1][c];
    if (((i + j + k) & 1) == 0) return old;  // black point keeps its value
    if (ZERO) return omega * (Fs[sf][r][c] / D);
    const T nb = E[se][r + 1][c - 1] + E[se][r + 1][c + 1] + E[se][r][c] + E[se][r + 2][c] + E[sl][r + 1][c] +
                 E[sh][r + 1][c];
    const T gs = (Fs[sf][r][c] + a * nb) / D;
    return (T(1) - omega) * old + omega * gs;
  };

  if (!ZERO) {
    fetch_e(z0 - 2);
    store_e(z0 - 2);
    fetch_e(z0 - 1);
    store_e(z0 - 1);
    fetch_e(z0);
  }
  fetch_f(z0 - 1);
  for (int k = z0 - 1; k <= z1; ++k) {
    if (!ZERO) store_e(k + 1);
    store_f(k);
    if (k < z1) {
      if (!ZERO) fetch_e(k + 2);
      fetch_f(k + 1);
    }
    __syncthreads();
    {  // red half-sweep on plane k over the tile and its one-point ring
      const int se = (k + 4) & 3, sl = (k + 3) & 3, sh = (k + 5) & 3, sf = (k + 3) % 3, smk = (k + 3) % 3;
      // a thread takes the row of its black half-sweep (row ty + 1) and the rows ty = 0, 1
      // the halo rows 0 and MY - 1: the black half-sweep of plane k-1 then reads red values
      // of plane k only at its own points, written here by the same thread
      for (int h = 0; h < 2; ++h) {
        int r;
        if (h == 0) {
          r = ty + 1;
        } else {
          if (ty >= 2) break;
          r = ty == 0 ? 0 : MY - 1;
        }
        const int c = 2 + 2 * tx;
        M[smk][r][c] = red_at(k, r, c, se, sl, sh, sf);
        M[smk][r][c + 1] = red_at(k, r, c + 1, se, sl, sh, sf);
      }
      if (tid < 2 * MY) {
        const int r = tid >> 1, c = (tid & 1) ? SX - 2 : 1;
        M[smk][r][c] = red_at(k, r, c, se, sl, sh, sf);
      }
    }
    // no barrier here: what crosses threads (the halo columns and rows of plane k, the red
    // values of planes k-1 and k-2) is read only after the barrier of the next plane
    const int kb = k - 1;  // black half-sweep on plane k-1 over the tile
    if (kb >= z0 && kb < z1) {
      const int s0 = (kb + 3) % 3, sl = (kb + 2) % 3, sh = (kb + 4) % 3, sf = (kb + 3) % 3, se = (kb + 4) & 3;
      const int j = y0 + ty, r = ty + 1;
      if (j < n && xi < n) {
        T v[2];
        for (int h = 0; h < 2; ++h) {
          const int c = 2 + 2 * tx + h, i = xi + h;
          if (i >= n) { v[h] = T(0); continue; }
          if (((i + j + kb) & 1) == 0) {
            const T nb = M[s0][r][c - 1] + M[s0][r][c + 1] + M[s0][r - 1][c] + M[s0][r + 1][c] + M[sl][r][c] +
                         M[sh][r][c];
            const T gs = (Fs[sf][r][c] + a * nb) / D;
            const T old = ZERO ? T(0) : E[se][r + 1][c];
            v[h] = (T(1) - omega) * old + omega * gs;
          } else {
            v[h] = M[s0][r][c];
          }
        }
        const long long o = kb * plane + (long long)j * g.pitch + xi;
        if (UPD) {
          double2 *up = (double2 *)(u + b * su + o);
          double2 w = *up;
          w.x += to_f64(v[0]);
          w.y += to_f64(v[1]);
          *up = w;
        } else {
          T2 w;
          w.x = v[0];
          w.y = v[1];
          *(T2 *)(eout + b * g.slab + o) = w;
        }
      }
    }
  }
}

// Full-row variant for n + 1 = NX in {64, 128, 256}: a tile spans the whole padded
// x row (the pad column is the zero wall), so no x ring is needed and no red point is
// computed twice in x.  Threads own x-pairs (one red, one black point each) across
// several rows; x neighbours come from the neighbouring lanes by warp shuffles.
constexpr int FTY = 8;               // output rows per tile
constexpr int FEY = FTY + 4;         // e_in rows (two-row ring)
constexpr int FMY = FTY + 2;         // red / f rows (one-row ring)

template <typename T, int NX, bool ZERO, bool UPD, int NT>
__global__ void __launch_bounds__(NT, 512 / NT * 2 > 4 ? 4 : 512 / NT * 2) rbgs_rows3d_kernel(Grid g, T a, T iD, T omega, const T *__restrict__ ein,
                                                             T *__restrict__ eout, const T *__restrict__ f,
                                                             double *__restrict__ u, long long su, int nzc, int zchunk) {
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  constexpr int NP = NX / 2;                  // pairs per row
  constexpr int RS = NT / NP;                 // rows covered per round of NT threads
  constexpr int PE = (FEY + RS - 1) / RS, PF = (FMY + RS - 1) / RS, PB = (FTY + RS - 1) / RS;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T2(*E)[FEY][NP] = (T2(*)[FEY][NP])sm_raw;                                         // [4][FEY][NP]
  T2(*M)[FMY][NP] = (T2(*)[FMY][NP])(sm_raw + sizeof(T2) * 4 * FEY * NP);             // [3][FMY][NP]
  T2(*Fs)[FMY][NP] = (T2(*)[FMY][NP])(sm_raw + sizeof(T2) * (4 * FEY + 3 * FMY) * NP);  // [3][FMY][NP]
  const int n = g.n, tid = threadIdx.x, px = tid % NP, ry = tid / NP, lane = tid & 31;
  const int y0 = blockIdx.y * FTY;
  const int zc = blockIdx.z % nzc, b = blockIdx.z / nzc;
  const int z0 = zc * zchunk, z1 = min(z0 + zchunk, n);
  const long long plane = (long long)g.ny * g.pitch;
  const T *Eb = ein + b * g.slab + 2 * px;
  const T *Fb = f + b * g.slab + 2 * px;
  const unsigned full = 0xffffffffu;

  T2 pe[PE], pf[PF];
  auto fetch = [&](const T *base, int k, int row0, int nrows, T2 *dst, int cnt) {
#pragma unroll
    for (int h = 0; h < cnt; ++h) {
      const int r = ry + RS * h, y = row0 + r;
      T2 v;
      v.x = T(0);
      v.y = T(0);
      if (r < nrows && k >= 0 && k < n && y >= 0 && y < n) v = *(const T2 *)(base + k * plane + (long long)y * g.pitch);
      dst[h] = v;
    }
  };
  auto store = [&](T2(*S)[NP], int nrows, const T2 *src, int cnt) {
#pragma unroll
    for (int h = 0; h < cnt; ++h) {
      const int r = ry + RS * h;
      if (r < nrows) S[r][px] = src[h];
    }
  };
  // x neighbours of the pair (c.x, c.y) in smem row `row`: left of c.x and right of
  // c.y, from the neighbouring lanes, or from shared memory at a warp edge (a row may
  // span several warps), or zero at the walls
  auto xnb = [&](T2 c, const T2 *row, T &left, T &right) {
    const T l = __shfl_up_sync(full, c.y, 1), r = __shfl_down_sync(full, c.x, 1);
    left = lane != 0 ? l : (px > 0 ? row[px - 1].y : T(0));
    right = lane != 31 ? r : (px < NP - 1 ? row[px + 1].x : T(0));
  };

  if (!ZERO) {
    fetch(Eb, z0 - 2, y0 - 2, FEY, pe, PE);
    store(E[(z0 + 2) & 3], FEY, pe, PE);
    fetch(Eb, z0 - 1, y0 - 2, FEY, pe, PE);
    store(E[(z0 + 3) & 3], FEY, pe, PE);
    fetch(Eb, z0, y0 - 2, FEY, pe, PE);
  }
  fetch(Fb, z0 - 1, y0 - 1, FMY, pf, PF);
  for (int k = z0 - 1; k <= z1; ++k) {
    if (!ZERO) store(E[(k + 5) & 3], FEY, pe, PE);
    store(Fs[(k + 3) % 3], FMY, pf, PF);
    if (k < z1) {
      if (!ZERO) fetch(Eb, k + 2, y0 - 2, FEY, pe, PE);
      fetch(Fb, k + 1, y0 - 1, FMY, pf, PF);
    }
    __syncthreads();
    {  // red half-sweep on plane k, rows y0-1 .. y0+FTY
      const int se = (k + 4) & 3, sl = (k + 3) & 3, sh = (k + 5) & 3, s3 = (k + 3) % 3;
      const bool kin = k >= 0 && k < n;
#pragma unroll
      for (int h = 0; h <= PB; ++h) {
        // the rows of the thread's black half-sweep, then the halo rows y0-1 and y0+FTY
        // (rows ry = 0, 1): the black half-sweep of plane k-1 reads red values of plane k
        // only at its own points, so no barrier separates the two half-sweeps
        int r;
        if (h < PB) {
          if (ry + RS * h >= FTY) continue;  // uniform per warp (a warp lies in one row)
          r = ry + RS * h + 1;
        } else {
          if (ry >= 2) continue;
          r = ry == 0 ? 0 : FMY - 1;
        }
        const int y = y0 - 1 + r;
        T2 out;
        out.x = T(0);
        out.y = T(0);
        const bool yin = kin && y >= 0 && y < n;
        if (ZERO) {
          const T2 fv = Fs[s3][r][px];
          const int ro = ((y + k) & 1) ? 0 : 1;   // red: x + y + k odd
          const int xr = 2 * px + ro;
          const T v = (yin && xr < n) ? omega * ((ro ? fv.y : fv.x) * iD) : T(0);
          if (ro) out.y = v; else out.x = v;
        } else {
          const T2 c = E[se][r + 1][px];
          T left, right;
          xnb(c, E[se][r + 1], left, right);
          if (yin) {
            const T2 up = E[se][r][px], dn = E[se][r + 2][px], zl = E[sl][r + 1][px], zh = E[sh][r + 1][px];
            const T2 fv = Fs[s3][r][px];
            const int ro = ((y + k) & 1) ? 0 : 1;
            out = c;
            const int xr = 2 * px + ro;
            if (xr < n) {
              T nb, fr, old;
              if (ro == 0) {
                nb = left + c.y + up.x + dn.x + zl.x + zh.x;
                fr = fv.x;
                old = c.x;
              } else {
                nb = c.x + right + up.y + dn.y + zl.y + zh.y;
                fr = fv.y;
                old = c.y;
              }
              const T gs = (fr + a * nb) * iD;
              const T v = omega == T(1) ? gs : old + omega * (gs - old);
              if (ro) out.y = v; else out.x = v;
            }
          }
        }
        M[s3][r][px] = out;
      }
    }
    const int kb = k - 1;  // black half-sweep on plane k-1, rows y0 .. y0+FTY-1
    if (kb >= z0 && kb < z1) {
      const int s0 = (kb + 3) % 3, sl = (kb + 2) % 3, sh = (kb + 4) % 3, se = (kb + 4) & 3;
#pragma unroll
      for (int h = 0; h < PB; ++h) {
        const int r = ry + RS * h;
        if (r >= FTY) break;
        const int y = y0 + r;
        const T2 c = M[s0][r + 1][px];
        T left, right;
        xnb(c, M[s0][r + 1], left, right);
        if (y >= n) continue;
        const T2 up = M[s0][r][px], dn = M[s0][r + 2][px], zl = M[sl][r + 1][px], zh = M[sh][r + 1][px];
        const T2 fv = Fs[s0][r + 1][px];
        const int bo = ((y + kb) & 1) ? 1 : 0;    // black: x + y + kb even
        T2 out = c;
        const int xb = 2 * px + bo;
        if (xb < n) {
          T nb, fr, old;
          if (bo == 0) {
            nb = left + c.y + up.x + dn.x + zl.x + zh.x;
            fr = fv.x;
            old = ZERO ? T(0) : E[se][r + 2][px].x;
          } else {
            nb = c.x + right + up.y + dn.y + zl.y + zh.y;
            fr = fv.y;
            old = ZERO ? T(0) : E[se][r + 2][px].y;
          }
          const T gs = (fr + a * nb) * iD;
          const T v = omega == T(1) ? gs : old + omega * (gs - old);
          if (bo) out.y = v; else out.x = v;
        }
        const long long o = kb * plane + (long long)y * g.pitch + 2 * px;
        if (UPD) {
          double2 *up2 = (double2 *)(u + b * su + o);
          double2 w = *up2;
          w.x += to_f64(out.x);
          w.y += to_f64(out.y);
          *up2 = w;
        } else {
          *(T2 *)(eout + b * g.slab + o) = out;
        }
      }
    }
  }
}

// residual + full weighting: coarse tile CTX x CTY, coarse z chunk CZC.  Fine smem
// column c <-> x = 2*I0 - 2 + c; the residual is needed on x in [2I0, 2I0+64] (c 2..66),
// e on x in [2I0-1, 2I0+65] (c 1..67); rows likewise with y.
constexpr int CTX = 32, CTY = 8, CZC = 16;
constexpr int QS = 2 * CTX + 4;           // smem row length (68)
constexpr int QY = 2 * CTY + 3;           // e rows: y in [2J0-1, 2J0+17]
constexpr int RYN = 2 * CTY + 1;          // residual rows: y in [2J0, 2J0+16]

template <typename T>
__global__ void __launch_bounds__(256, 4) resrestrict3d_kernel(Grid gf, Grid gc, T a, const T *__restrict__ e,
                                                               const T *__restrict__ f, T *__restrict__ fc, int nzc) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T(*E)[QY][QS] = (T(*)[QY][QS])sm_raw;                                  // [4][QY][QS]
  T(*Fs)[QS] = (T(*)[QS])(sm_raw + sizeof(T) * 4 * QY * QS);             // [RYN][QS]
  T(*R)[QS] = (T(*)[QS])(sm_raw + sizeof(T) * (4 * QY + RYN) * QS);      // [RYN][QS]
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  const int n = gf.n, nc = gc.n, tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int I0 = blockIdx.x * CTX, J0 = blockIdx.y * CTY;
  const int zc = blockIdx.z % nzc, b = blockIdx.z / nzc;
  const int K0 = zc * CZC, K1 = min(K0 + CZC, nc);
  const int fx = 2 * I0 - 2, fy = 2 * J0 - 1;  // x of smem column 0, y of e row 0
  const long long plane = (long long)gf.ny * gf.pitch, cplane = (long long)gc.ny * gc.pitch;
  const T *Eb = e + b * gf.slab;
  const T *Fb = f + b * gf.slab;
  const int xi = 2 * I0 + 2 * tx;  // pair x of this thread (smem column 2 + 2 tx)
  // halo: e columns {1, 66, 67} x QY rows; f column 66 x RYN rows
  const int eh_row = tid / 3, eh_col = (tid % 3) == 0 ? 1 : 65 + (tid % 3);
  const bool has_eh = tid < 3 * QY, has_fh = tid >= 64 && tid < 64 + RYN;
  T2 pe[3], pf[3];
  T pe_h = T(0), pf_h = T(0);
  auto pair = [&](const T *base, int k, int j) -> T2 {
    T2 v;
    v.x = T(0);
    v.y = T(0);
    if (k >= 0 && k < n && j >= 0 && j < n && xi < n) v = *(const T2 *)(base + k * plane + (long long)j * gf.pitch + xi);
    return v;
  };
  auto one = [&](const T *base, int k, int j, int i) -> T {
    return (k >= 0 && k < n && j >= 0 && j < n && i >= 0 && i < n) ? base[k * plane + (long long)j * gf.pitch + i] : T(0);
  };
  auto fetch_e = [&](int k) {
    for (int h = 0; h < 3; ++h)
      if (ty + 8 * h < QY) pe[h] = pair(Eb, k, fy + ty + 8 * h);
    if (has_eh) pe_h = one(Eb, k, fy + eh_row, fx + eh_col);
  };
  auto fetch_f = [&](int k) {
    for (int h = 0; h < 3; ++h)
      if (ty + 8 * h < RYN) pf[h] = pair(Fb, k, fy + 1 + ty + 8 * h);
    if (has_fh) pf_h = one(Fb, k, fy + 1 + (tid - 64), fx + 66);
  };
  auto store_e = [&](int k) {
    T(*S)[QS] = E[(k + 4) & 3];
    for (int h = 0; h < 3; ++h)
      if (ty + 8 * h < QY) *(T2 *)&S[ty + 8 * h][2 + 2 * tx] = pe[h];
    if (has_eh) S[eh_row][eh_col] = pe_h;
  };
  auto store_f = [&]() {
    for (int h = 0; h < 3; ++h)
      if (ty + 8 * h < RYN) *(T2 *)&Fs[ty + 8 * h][2 + 2 * tx] = pf[h];
    if (has_fh) Fs[tid - 64][66] = pf_h;
  };
  // residual at fine plane z, smem residual row rr (y = fy + 1 + rr), column c
  auto resid = [&](int rr, int c, int s0, int sl, int sh) -> T {
    const int i = fx + c, j = fy + 1 + rr;
    if (i >= n || j >= n) return T(0);
    const int er = rr + 1;
    const T ec = E[s0][er][c];
    const T nb = E[s0][er][c - 1] + E[s0][er][c + 1] + E[s0][er - 1][c] + E[s0][er + 1][c] + E[sl][er][c] +
                 E[sh][er][c];
    return Fs[rr][c] - (ec - a * (nb - T(6) * ec));
  };
  const int cx = tid % CTX, cy = tid / CTX;
  T acc = T(0);
  const int zb = 2 * K0, ze = 2 * K1;  // fine planes 2K .. 2K+2 feed coarse plane K
  fetch_e(zb - 1);
  store_e(zb - 1);
  fetch_e(zb);
  store_e(zb);
  fetch_e(zb + 1);
  fetch_f(zb);
  for (int z = zb; z <= ze; ++z) {
    store_e(z + 1);  // ring slot of plane z-3, unused
    store_f();       // plane z
    if (z < ze) {    // next planes in flight during this plane's work
      fetch_e(z + 2);
      fetch_f(z + 1);
    }
    __syncthreads();
    const int s0 = (z + 4) & 3, sl = (z + 3) & 3, sh = (z + 5) & 3;
    for (int rr = ty; rr < RYN; rr += 8) {
      R[rr][2 + 2 * tx] = resid(rr, 2 + 2 * tx, s0, sl, sh);
      R[rr][3 + 2 * tx] = resid(rr, 3 + 2 * tx, s0, sl, sh);
    }
    if (tid >= 128 && tid < 128 + RYN) R[tid - 128][66] = resid(tid - 128, 66, s0, sl, sh);
    __syncthreads();
    // x-y full weighting of this fine plane at the thread's coarse point:
    // fine x = 2I+1 is column 2cx+3, fine y = 2J+1 is residual row 2cy+1
    const int c0 = 2 * cx + 3, r0 = 2 * cy + 1;
    const T rxy = T(0.25) * (T(0.25) * R[r0 - 1][c0 - 1] + T(0.5) * R[r0 - 1][c0] + T(0.25) * R[r0 - 1][c0 + 1]) +
                  T(0.5) * (T(0.25) * R[r0][c0 - 1] + T(0.5) * R[r0][c0] + T(0.25) * R[r0][c0 + 1]) +
                  T(0.25) * (T(0.25) * R[r0 + 1][c0 - 1] + T(0.5) * R[r0 + 1][c0] + T(0.25) * R[r0 + 1][c0 + 1]);
    const int I = I0 + cx, J = J0 + cy;
    if ((z & 1) == 0) {
      if (z > zb && I < nc && J < nc) fc[b * gc.slab + (z / 2 - 1) * cplane + (long long)J * gc.pitch + I] = acc + T(0.25) * rxy;
      acc = T(0.25) * rxy;
    } else {
      acc += T(0.5) * rxy;
    }
  }
}

// e (fine) += P e_c: thread per coarse cell (1-based J covers fine 2J+1 and 2J+2)
template <typename T>
__global__ void prolong3d_kernel(Grid gf, Grid gc, const T *__restrict__ ec, T *__restrict__ e, int batch) {
  const int nc = gc.n, n = gf.n;
  const int J = blockIdx.x * blockDim.x + threadIdx.x;   // 0..nc
  const int K = blockIdx.y * blockDim.y + threadIdx.y;   // 0..nc
  const int L = blockIdx.z % (nc + 1), b = blockIdx.z / (nc + 1);
  if (J > nc || K > nc || b >= batch) return;
  const T *C = ec + b * gc.slab;
  const long long cpl = (long long)gc.ny * gc.pitch;
  // corners: coarse 1-based J..J+1 (0 and nc+1 are walls)
  T c[2][2][2];
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int X = J + dx, Y = K + dy, Z = L + dz;
        c[dz][dy][dx] = (X >= 1 && X <= nc && Y >= 1 && Y <= nc && Z >= 1 && Z <= nc)
                            ? C[(Z - 1) * cpl + (long long)(Y - 1) * gc.pitch + (X - 1)]
                            : T(0);
      }
  T *Eb = e + b * gf.slab;
  const long long pl = (long long)gf.ny * gf.pitch;
  // fine 0-based index 2J is the mid point (weights 1/2, 1/2), 2J+1 is coarse J+1
  for (int pz = 0; pz < 2; ++pz) {
    const int k = 2 * L + pz;
    if (k >= n) continue;
    for (int py = 0; py < 2; ++py) {
      const int j = 2 * K + py;
      if (j >= n) continue;
      for (int px = 0; px < 2; ++px) {
        const int i = 2 * J + px;
        if (i >= n) continue;
        T v = T(0);
        for (int dz = 0; dz < 2; ++dz) {
          const T wz = pz == 0 ? T(0.5) : (dz == 1 ? T(1) : T(0));
          if (wz == T(0)) continue;
          for (int dy = 0; dy < 2; ++dy) {
            const T wy = py == 0 ? T(0.5) : (dy == 1 ? T(1) : T(0));
            if (wy == T(0)) continue;
            for (int dx = 0; dx < 2; ++dx) {
              const T wx = px == 0 ? T(0.5) : (dx == 1 ? T(1) : T(0));
              if (wx == T(0)) continue;
              v += wx * wy * wz * c[dz][dy][dx];
            }
          }
        }
        Eb[k * pl + (long long)j * gf.pitch + i] += v;
      }
    }
  }
}

template <typename T, int NX, bool ZERO, bool UPD, int NT>
void launch_rows(const Launch &L, const Grid &g, T a, T D, T omega, const void *ein, void *eout, const void *f,
                 double *u, long long su, int batch, int zchunk) {
  const T iD = T(1) / D;
  using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
  const size_t smem = sizeof(T2) * (4 * FEY + 6 * FMY) * (NX / 2);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(rbgs_rows3d_kernel<T, NX, ZERO, UPD, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  if (zchunk <= 0) zchunk = RZC;
  const int nty = (g.n + FTY - 1) / FTY, nzc = (g.n + zchunk - 1) / zchunk;
  dim3 gr(1, nty, nzc * batch);
  rbgs_rows3d_kernel<T, NX, ZERO, UPD, NT><<<gr, NT, smem, L.stream>>>(g, a, iD, omega, (const T *)ein, (T *)eout,
                                                                        (const T *)f, u, su, nzc, zchunk);
}

template <typename T, bool ZERO, bool UPD>
void launch_sweep(const Launch &L, const Grid &g, double c, double omega, const void *ein, void *eout, const void *f,
                  double *u, long long su, int batch, int zchunk, int threads) {
  const T a = (T)(c * g.ih2), D = T(1) + T(6) * a;
  const bool wide = threads >= 512;
  if (g.pitch == 256) {
    if (wide) return launch_rows<T, 256, ZERO, UPD, 512>(L, g, a, D, (T)omega, ein, eout, f, u, su, batch, zchunk);
    return launch_rows<T, 256, ZERO, UPD, 256>(L, g, a, D, (T)omega, ein, eout, f, u, su, batch, zchunk);
  }
  if (g.pitch == 128) {
    if (wide) return launch_rows<T, 128, ZERO, UPD, 512>(L, g, a, D, (T)omega, ein, eout, f, u, su, batch, zchunk);
    return launch_rows<T, 128, ZERO, UPD, 256>(L, g, a, D, (T)omega, ein, eout, f, u, su, batch, zchunk);
  }
  if (g.pitch == 64) return launch_rows<T, 64, ZERO, UPD, 256>(L, g, a, D, (T)omega, ein, eout, f, u, su, batch, zchunk);
  if (zchunk <= 0) zchunk = RZC;
  const int ntx = (g.n + RTX - 1) / RTX, nty = (g.n + RTY - 1) / RTY, nzc = (g.n + zchunk - 1) / zchunk;
  const size_t smem = sizeof(T) * (4 * EY + 6 * MY) * SX;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(rbgs_sweep3d_kernel<T, ZERO, UPD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  dim3 gr(ntx, nty, nzc * batch);
  rbgs_sweep3d_kernel<T, ZERO, UPD><<<gr, 256, smem, L.stream>>>(g, a, D, (T)omega, (const T *)ein, (T *)eout,
                                                                  (const T *)f, u, su, nzc, zchunk);
}

}  // namespace

bool rbgs_rows_supported(const Grid &g) {
  return g.dim == 3 && (g.pitch == 256 || g.pitch == 128 || g.pitch == 64);
}

cudaError_t k_rbgs_sweep3d(const Launch &L, const Grid &g, double c, double omega, Prec pr, const void *ein,
                           void *eout, const void *f, double *u, long long su, int batch, bool zero, bool update_u,
                           int zchunk, int threads) {
  Scope sc(L, zero ? K_RBGS3D_ZERO : (update_u ? K_RBGS3D_UPD : K_RBGS3D), g, batch, pr);
  if (pr == F32) {
    if (zero && update_u) launch_sweep<float, true, true>(L, g, c, omega, ein, eout, f, u, su, batch, zchunk, threads);
    else if (zero) launch_sweep<float, true, false>(L, g, c, omega, ein, eout, f, u, su, batch, zchunk, threads);
    else if (update_u) launch_sweep<float, false, true>(L, g, c, omega, ein, eout, f, u, su, batch, zchunk, threads);
    else launch_sweep<float, false, false>(L, g, c, omega, ein, eout, f, u, su, batch, zchunk, threads);
  } else {
    if (zero && update_u) launch_sweep<double, true, true>(L, g, c, omega, ein, eout, f, u, su, batch, zchunk, threads);
    else if (zero) launch_sweep<double, true, false>(L, g, c, omega, ein, eout, f, u, su, batch, zchunk, threads);
    else if (update_u) launch_sweep<double, false, true>(L, g, c, omega, ein, eout, f, u, su, batch, zchunk, threads);
    else launch_sweep<double, false, false>(L, g, c, omega, ein, eout, f, u, su, batch, zchunk, threads);
  }
  return sc.done();
}

template <typename T>
void launch_resrestrict(const Launch &L, const Grid &gf, const Grid &gc, double c, const void *e, const void *f,
                        void *fc, int batch) {
  const int ntx = (gc.n + CTX - 1) / CTX, nty = (gc.n + CTY - 1) / CTY, nzc = (gc.n + CZC - 1) / CZC;
  const size_t smem = sizeof(T) * (4 * QY + 2 * RYN) * QS;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(resrestrict3d_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  dim3 gr(ntx, nty, nzc * batch);
  resrestrict3d_kernel<T><<<gr, 256, smem, L.stream>>>(gf, gc, (T)(c * gf.ih2), (const T *)e, (const T *)f, (T *)fc,
                                                       nzc);
}

cudaError_t k_resrestrict3d(const Launch &L, const Grid &gf, const Grid &gc, double c, Prec pr, const void *e,
                            const void *f, void *fc, int batch) {
  Scope sc(L, K_RESRESTRICT3D, gc, batch, pr);
  if (pr == F32) launch_resrestrict<float>(L, gf, gc, c, e, f, fc, batch);
  else launch_resrestrict<double>(L, gf, gc, c, e, f, fc, batch);
  return sc.done();
}

cudaError_t k_prolong3d(const Launch &L, const Grid &gf, const Grid &gc, Prec pr, const void *ec, void *e, int batch) {
  Scope sc(L, K_PROLONG3D, gf, batch, pr);
  const int m = gc.n + 1;
  dim3 bl(32, 8, 1);
  dim3 gr((m + 31) / 32, (m + 7) / 8, m * batch);
  if (pr == F32)
    prolong3d_kernel<float><<<gr, bl, 0, L.stream>>>(gf, gc, (const float *)ec, (float *)e, batch);
  else
    prolong3d_kernel<double><<<gr, bl, 0, L.stream>>>(gf, gc, (const double *)ec, (double *)e, batch);
  return sc.done();
}

}  // namespace pmg
