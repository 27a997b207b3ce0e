// learned.cu -- convolutional multigrid correction network: forward, backward, Adam,
// synthetic training pairs, and the correction step inside a V-cycle.
//
// The network (the paper has no learned component; this is an extension of its
// multigrid sub-step solver):
//   y = W3 * relu(W2 * relu(W1 * x + b1) + b2) + b3,
// three 3x3x3 convolutions with zero padding on the interior grid, channels
// 1 -> 16 -> 16 -> 1.  On a multigrid level with operator I - c Lap_h and diagonal
// D = 1 + 6 c / h^2, the input is the scaled residual x = D^-1 (f - (I - c Lap_h) e)
// and y is added to the correction e; it replaces the second pre-smoothing sweep.
// Training minimises 0.5 mean((Ahat^p (y - t))^2) with Ahat = D^-1 (I - c Lap_h) =
// I - kappa N (N: sum of the 6 face neighbours, kappa = (c/h^2) / D), t the exact
// remaining error and p in 0..3: p = 1 is the scaled residual the correction leaves,
// p = 2 weights every error mode by its squared eigenvalue of Ahat, so that smooth
// modes, which the coarse-grid correction removes, do not count.
//
// Weights are kept in FP32 and used in BF16 by the tensor-core layer; activations are
// stored in BF16, every sum is accumulated in FP32.
//
// The 16 -> 16 layer is an implicit GEMM on the tensor cores (mma.sync m16n8k16, BF16
// in, FP32 accumulate): a warp takes 16 consecutive points of one grid row as M, the
// 16 output channels as N (two 8-wide tiles) and the 27 taps x 16 input channels as K
// (one k16 step per tap).  The same kernel with the transposed, tap-flipped weights
// gives the input gradient of the backward pass.  The 1 -> 16 and 16 -> 1 layers and
// the weight-gradient reductions run on the FP32 cores.
#include <cmath>

#include "pmg_internal.cuh"

namespace pmg {
namespace {

constexpr int NC = kNetC;

__device__ __forceinline__ void tap_offset(int t, int &dz, int &dy, int &dx) {
  dz = t / 9 - 1;
  dy = (t / 3) % 3 - 1;
  dx = t % 3 - 1;
}

// point (b, z, y, x) of dense [batch][n][n][n] storage
__device__ __forceinline__ long long dense_index(int b, int z, int y, int x, int n) {
  return (((long long)b * n + z) * n + y) * n + x;
}

// point (b, z, y, x) of a grid function in the layout of g (pitch / slab)
__device__ __forceinline__ long long io_index(const NetGrid &g, int b, int z, int y, int x) {
  return b * g.slab + ((long long)z * g.n + y) * g.pitch + x;
}

__device__ __forceinline__ bool inside(int z, int y, int x, int n) {
  return z >= 0 && z < n && y >= 0 && y < n && x >= 0 && x < n;
}

__device__ __forceinline__ void split_point(long long p, int n, int &b, int &z, int &y, int &x) {
  x = (int)(p % n);
  y = (int)((p / n) % n);
  z = (int)((p / ((long long)n * n)) % n);
  b = (int)(p / ((long long)n * n * n));
}

// splitmix64 finaliser (Steele, Lea, Flood 2014) as a counter-based generator:
// value i of stream `seed` = mix(seed + (i + 1) * golden gamma)
__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ double uniform01(unsigned long long seed, unsigned long long i) {
  return (double)(mix64(seed + (i + 1) * 0x9e3779b97f4a7c15ULL) >> 11) * (1.0 / 9007199254740992.0);
}

int grid_blocks(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

Grid cube(int n) { return make_grid(3, n); }

// ---------------------------------------------------------------- layer 1 (1 -> 16)
__global__ void l1_fwd_kernel(NetGrid g, const float *__restrict__ x, const float *__restrict__ prm,
                              __nv_bfloat16 *__restrict__ a1) {
  __shared__ float W[NC * 27 + NC];  // W1 then b1
  for (int i = threadIdx.x; i < NC * 27 + NC; i += blockDim.x) W[i] = prm[kNetW1 + i];
  __syncthreads();
  const long long npts = (long long)g.batch * g.n * g.n * g.n;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x) {
    int b, z, y, xx;
    split_point(p, g.n, b, z, y, xx);
    float acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = W[NC * 27 + c];
    for (int t = 0; t < 27; ++t) {
      int dz, dy, dx;
      tap_offset(t, dz, dy, dx);
      if (!inside(z + dz, y + dy, xx + dx, g.n)) continue;
      const float v = x[io_index(g, b, z + dz, y + dy, xx + dx)];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] += W[c * 27 + t] * v;
    }
    __nv_bfloat162 *o = (__nv_bfloat162 *)(a1 + p * NC);
#pragma unroll
    for (int c = 0; c < NC; c += 2) o[c / 2] = __floats2bfloat162_rn(fmaxf(acc[c], 0.f), fmaxf(acc[c + 1], 0.f));
  }
}

// ---------------------------------------------------------------- layer 2 (16 -> 16), tensor cores
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// out[p][o] = sum_t sum_c Wb[t][o][c] act[p + off_t][c]   (Wb: BF16 [27][16][16])
// MODE 0 (forward):  out_bf[p][o] = relu(. + bias[o])               (BF16)
// MODE 1 (backward): out_f[p][o]  = . if mask[p][o] > 0, else 0      (FP32)
// An implicit GEMM on mma.sync m16n8k16 (BF16 in, FP32 accumulate): M = 16 consecutive
// points of a grid row, N = 16 output channels (two 8-wide tiles), K = 27 taps x 16
// input channels (one k16 step per tap).  Fragment layout (PTX ISA, "Matrix Fragments
// for mma.m16n8k16"), g = lane / 4, q = lane % 4: A registers 0..3 hold (row g, k
// 2q..2q+1), (row g+8, k 2q..), (row g, k 2q+8..), (row g+8, k 2q+8..); B registers 0..1
// hold (k 2q..2q+1, col g), (k 2q+8..2q+9, col g); C holds (row g, col 2q..2q+1) and
// (row g+8, col 2q..2q+1).  Rows = points, k = input channel, col = output channel.
//
// A CTA takes tiles of 16 (x) x 8 (y) x 4 (z) points and stages their 18 x 10 x 6
// neighbourhood in shared memory once (zeros outside the grid, so no tap needs a bounds
// check), each point's 16 channels split into two 16-byte halves (channels 0-7, 8-15) in
// separate arrays, so that the eight rows of an 8 x 8 ldmatrix operand are 128
// contiguous bytes (no bank conflicts).  Per tap a warp loads the B operands of both
// N tiles with one ldmatrix.x4 from the staged weights (same half split) and, for each of
// its four 16-point rows, the A operand with one ldmatrix.x4: matrices (points 0-7,
// channels 0-7), (points 8-15, ch 0-7), (points 0-7, ch 8-15), (points 8-15, ch 8-15)
// are A registers 0..3 (ldmatrix gives thread (g, q) row g, elements 2q, 2q+1 of each
// matrix).
constexpr int L2X = 16, L2Y = 8, L2Z = 4;                                 // tile
constexpr int L2HX = L2X + 2, L2HY = L2Y + 2, L2HZ = L2Z + 2;               // with halo
constexpr int L2HP = L2HX * L2HY * L2HZ;                                    // staged points

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"((unsigned)__cvta_generic_to_shared(p)));
}

template <int MODE>
__global__ void __launch_bounds__(256) l2_tile_kernel(NetGrid g, const __nv_bfloat16 *__restrict__ act,
                                                      const __nv_bfloat16 *__restrict__ Wb,
                                                      const float *__restrict__ bias,
                                                      const __nv_bfloat16 *__restrict__ mask,
                                                      __nv_bfloat16 *__restrict__ out_bf, float *__restrict__ out_f) {
  __shared__ __align__(128) uint4 Wh[2][27][NC];   // [channel half][tap][output channel]
  __shared__ __align__(128) uint4 Ah[2][L2HP];     // [channel half][staged point]
  for (int i = threadIdx.x; i < 27 * NC * 2; i += blockDim.x) {
    const int half = i & 1, to = i >> 1;  // to = t * NC + o
    Wh[half][to / NC][to % NC] = ((const uint4 *)Wb)[i];
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, t4 = lane & 3;
  // this lane's ldmatrix row: matrix lane / 8, row lane % 8
  const int mat = lane >> 3, mrow = lane & 7;
  const int a_pt = (mat & 1) * 8 + mrow, a_half = mat >> 1;  // A: point of the row segment, channel half
  const int b_half = mat & 1, b_o = (mat >> 1) * 8 + mrow;   // B: channel half, output channel
  const int ntx = (g.n + L2X - 1) / L2X, nty = (g.n + L2Y - 1) / L2Y, ntz = (g.n + L2Z - 1) / L2Z;
  const long long ntiles = (long long)g.batch * ntx * nty * ntz;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int tx = (int)(tile % ntx), ty = (int)((tile / ntx) % nty), tz = (int)((tile / ((long long)ntx * nty)) % ntz);
    const int b = (int)(tile / ((long long)ntx * nty * ntz));
    const int x0 = tx * L2X, y0 = ty * L2Y, z0 = tz * L2Z;
    __syncthreads();  // the previous tile's reads are done (and the weights staged)
    for (int q = threadIdx.x; q < L2HP; q += blockDim.x) {  // one point (both halves) per thread
      const int xx = x0 - 1 + q % L2HX, yy = y0 - 1 + (q / L2HX) % L2HY, zz = z0 - 1 + q / (L2HX * L2HY);
      uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
      if (inside(zz, yy, xx, g.n)) {
        const uint4 *src = (const uint4 *)(act + dense_index(b, zz, yy, xx, g.n) * NC);
        lo = src[0];
        hi = src[1];
      }
      Ah[0][q] = lo;
      Ah[1][q] = hi;
    }
    __syncthreads();
    float acc[4][2][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][nt][q] = 0.f;
#pragma unroll 1
    for (int t = 0; t < 27; ++t) {
      int dz, dy, dx;
      tap_offset(t, dz, dy, dx);
      unsigned bf[4];
      ldsm_x4(bf, &Wh[b_half][t][b_o]);
      const unsigned b0[2] = {bf[0], bf[1]}, b1[2] = {bf[2], bf[3]};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = warp + 8 * r, yl = row % L2Y, zl = row / L2Y;  // the warp's rows of the tile
        const int q = ((zl + dz + 1) * L2HY + (yl + dy + 1)) * L2HX + (dx + 1) + a_pt;
        unsigned a[4];
        ldsm_x4(a, &Ah[a_half][q]);
        mma_bf16(acc[r][0], a, b0);
        mma_bf16(acc[r][1], a, b1);
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int row = warp + 8 * r, y = y0 + row % L2Y, z = z0 + row / L2Y;
      if (y >= g.n || z >= g.n) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int x = x0 + gq + 8 * h;
        if (x >= g.n) continue;
        const long long p = dense_index(b, z, y, x, g.n);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const int o = nt * 8 + 2 * t4;
          float v0 = acc[r][nt][2 * h], v1 = acc[r][nt][2 * h + 1];
          if (MODE == 0) {
            v0 = fmaxf(v0 + bias[o], 0.f);
            v1 = fmaxf(v1 + bias[o + 1], 0.f);
            *(__nv_bfloat162 *)(out_bf + p * NC + o) = __floats2bfloat162_rn(v0, v1);
          } else {
            const float2 m = __bfloat1622float2(*(const __nv_bfloat162 *)(mask + p * NC + o));
            *(float2 *)(out_f + p * NC + o) = make_float2(m.x > 0.f ? v0 : 0.f, m.y > 0.f ? v1 : 0.f);
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------- layer 3 (16 -> 1)
// y = b3 + sum_t sum_c W3[t][c] a2[p + off_t][c];  out (+)= y in the layout of g
template <typename TO, bool ADD>
__global__ void l3_fwd_kernel(NetGrid g, const __nv_bfloat16 *__restrict__ a2, const float *__restrict__ prm,
                              TO *__restrict__ out) {
  __shared__ float W[27 * NC + 1];  // W3 then b3
  for (int i = threadIdx.x; i < 27 * NC + 1; i += blockDim.x) W[i] = prm[kNetW3 + i];
  __syncthreads();
  const long long npts = (long long)g.batch * g.n * g.n * g.n;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x) {
    int b, z, y, x;
    split_point(p, g.n, b, z, y, x);
    float acc = W[27 * NC];
    for (int t = 0; t < 27; ++t) {
      int dz, dy, dx;
      tap_offset(t, dz, dy, dx);
      if (!inside(z + dz, y + dy, x + dx, g.n)) continue;
      const __nv_bfloat162 *r = (const __nv_bfloat162 *)(a2 + dense_index(b, z + dz, y + dy, x + dx, g.n) * NC);
#pragma unroll
      for (int c = 0; c < NC; c += 2) {
        const float2 v = __bfloat1622float2(r[c / 2]);
        acc += W[t * NC + c] * v.x + W[t * NC + c + 1] * v.y;
      }
    }
    const long long o = io_index(g, b, z, y, x);
    if (ADD) out[o] += (TO)acc;
    else out[o] = (TO)acc;
  }
}

// ---------------------------------------------------------------- loss and backward
// sum of the 6 face neighbours of v (dense storage, zero outside)
__device__ __forceinline__ float nb6(const float *__restrict__ v, int b, int z, int y, int x, int n) {
  float s = 0.f;
  if (x > 0) s += v[dense_index(b, z, y, x - 1, n)];
  if (x < n - 1) s += v[dense_index(b, z, y, x + 1, n)];
  if (y > 0) s += v[dense_index(b, z, y - 1, x, n)];
  if (y < n - 1) s += v[dense_index(b, z, y + 1, x, n)];
  if (z > 0) s += v[dense_index(b, z - 1, y, x, n)];
  if (z < n - 1) s += v[dense_index(b, z + 1, y, x, n)];
  return s;
}

// d = y - t (stored), for the next kernel
__global__ void net_diff_kernel(long long npts, const float *__restrict__ y, const float *__restrict__ t,
                                float *__restrict__ d) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x)
    d[p] = y[p] - t[p];
}

// out = scale * Ahat v (scale * v for kappa = 0)
__global__ void net_ahat_kernel(NetGrid g, const float *__restrict__ v, const float *__restrict__ kappa, float scale,
                                float *__restrict__ out) {
  const long long npts = (long long)g.batch * g.n * g.n * g.n;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x) {
    int b, z, y, x;
    split_point(p, g.n, b, z, y, x);
    out[p] = scale * (v[p] - kappa[b] * nb6(v, b, z, y, x, g.n));
  }
}

// loss += 0.5 sum w^2 / count
__global__ void net_sqloss_kernel(long long npts, const float *__restrict__ w, double inv_count,
                                  double *__restrict__ loss) {
  double acc = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x)
    acc += 0.5 * (double)w[p] * w[p] * inv_count;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

__global__ void net_scale_kernel(long long npts, const float *__restrict__ v, float scale, float *__restrict__ out) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x)
    out[p] = scale * v[p];
}

// gz2[p][c] = (a2[p][c] > 0) sum_t W3[t][c] gy[p - off_t], stored in FP32 and BF16
__global__ void l3_bwd_data_kernel(NetGrid g, const float *__restrict__ gy, const __nv_bfloat16 *__restrict__ a2,
                                   const float *__restrict__ prm, float *__restrict__ gz2,
                                   __nv_bfloat16 *__restrict__ gz2b) {
  __shared__ float W[27 * NC];
  for (int i = threadIdx.x; i < 27 * NC; i += blockDim.x) W[i] = prm[kNetW3 + i];
  __syncthreads();
  const long long npts = (long long)g.batch * g.n * g.n * g.n;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x) {
    int b, z, y, x;
    split_point(p, g.n, b, z, y, x);
    float acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.f;
    for (int t = 0; t < 27; ++t) {
      int dz, dy, dx;
      tap_offset(t, dz, dy, dx);
      if (!inside(z - dz, y - dy, x - dx, g.n)) continue;
      const float v = gy[dense_index(b, z - dz, y - dy, x - dx, g.n)];
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] += W[t * NC + c] * v;
    }
    const __nv_bfloat162 *m = (const __nv_bfloat162 *)(a2 + p * NC);
#pragma unroll
    for (int c = 0; c < NC; c += 2) {
      const float2 mv = __bfloat1622float2(m[c / 2]);
      const float v0 = mv.x > 0.f ? acc[c] : 0.f, v1 = mv.y > 0.f ? acc[c + 1] : 0.f;
      *(float2 *)(gz2 + p * NC + c) = make_float2(v0, v1);
      *(__nv_bfloat162 *)(gz2b + p * NC + c) = __floats2bfloat162_rn(v0, v1);
    }
  }
}

// weight and bias gradients of one layer: dW[o][t][c] += sum_p gsrc[p][o] a[p + off_t][c],
// db[o] += sum_p gsrc[p][o] (all dense).  A CTA walks 32-point row segments; thread j
// owns the outputs j, j + 256, ...; the 3 x 3 rows x 34 points neighbourhood of a
// segment is staged in shared memory; every CTA adds its partial sums once at the end.
template <int CO, int CI, typename TA>
__global__ void __launch_bounds__(256) wgrad_kernel(NetGrid g, const float *__restrict__ gsrc,
                                                    const TA *__restrict__ a, float *__restrict__ dW,
                                                    float *__restrict__ db) {
  constexpr int NOUT = CO * 27 * CI, PER = (NOUT + 255) / 256;
  __shared__ float Gs[32][CO];
  __shared__ float As[9][34][CI];
  float acc[PER];
  float bacc = 0.f;
#pragma unroll
  for (int k = 0; k < PER; ++k) acc[k] = 0.f;
  const int segs = (g.n + 31) / 32;
  const long long nseg = (long long)g.batch * g.n * g.n * segs;
  for (long long s = blockIdx.x; s < nseg; s += gridDim.x) {
    const int seg = (int)(s % segs);
    const long long row = s / segs;
    const int y = (int)(row % g.n), z = (int)((row / g.n) % g.n), b = (int)(row / ((long long)g.n * g.n));
    const int x0 = seg * 32;
    __syncthreads();  // the previous segment's reads are done
    for (int i = threadIdx.x; i < 32 * CO; i += blockDim.x) {
      const int xi = i / CO, o = i % CO, x = x0 + xi;
      Gs[xi][o] = x < g.n ? gsrc[dense_index(b, z, y, x, g.n) * CO + o] : 0.f;
    }
    for (int i = threadIdx.x; i < 9 * 34 * CI; i += blockDim.x) {
      const int c = i % CI, xi = (i / CI) % 34, r = i / (CI * 34);
      const int zz = z + r / 3 - 1, yy = y + r % 3 - 1, xx = x0 + xi - 1;
      As[r][xi][c] = inside(zz, yy, xx, g.n) ? (float)a[dense_index(b, zz, yy, xx, g.n) * CI + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int j = threadIdx.x + 256 * k;
      if (j < NOUT) {
        const int c = j % CI, t = (j / CI) % 27, o = j / (CI * 27);
        const int r = (t / 9) * 3 + (t / 3) % 3, dx = t % 3;  // (dz, dy) row and x offset + 1
        float sum = 0.f;
        for (int xi = 0; xi < 32; ++xi) sum += Gs[xi][o] * As[r][xi + dx][c];
        acc[k] += sum;
      }
    }
    if (threadIdx.x < CO)
      for (int xi = 0; xi < 32; ++xi) bacc += Gs[xi][threadIdx.x];
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int j = threadIdx.x + 256 * k;
    if (j < NOUT) atomicAdd(dW + j, acc[k]);
  }
  if (threadIdx.x < CO) atomicAdd(db + threadIdx.x, bacc);
}

// 16 -> 16 weight gradient on the tensor cores: for every tap t,
//   dW[o][t][c] += sum_p G[p][o] act[p + off_t][c]
// is a GEMM with M = o (16), N = c (two 8-wide tiles) and K = grid points.  A CTA walks
// 32-point row segments: it stages G transposed (Gt[o][x], BF16) and the 3 x 3 rows x
// 34 points neighbourhood of the activations transposed (At[row][c][x], BF16) in shared
// memory, so that both mma operands have their K (point) pairs adjacent; warp w owns
// the taps w, w + 8, w + 16, w + 24 and keeps their 16 x 16 sums in registers (FP32),
// added to dW once per CTA.  db[o] += sum_p G[p][o] in FP32.
__global__ void __launch_bounds__(256) wgrad_mma_kernel(NetGrid g, const float *__restrict__ G,
                                                        const __nv_bfloat16 *__restrict__ act, float *__restrict__ dW,
                                                        float *__restrict__ db) {
  constexpr int XS = 40;  // row pitch (elements) of the staged tiles: 34 used, padded against bank conflicts
  __shared__ __align__(16) __nv_bfloat16 Gt[NC][XS];
  __shared__ __align__(16) __nv_bfloat16 At[9][NC][XS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, t4 = lane & 3;
  float acc[4][2][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[j][nt][q] = 0.f;
  float bacc = 0.f;  // bias sum of channel threadIdx.x % 16
  const int segs = (g.n + 31) / 32;
  const long long nseg = (long long)g.batch * g.n * g.n * segs;
  for (long long s = blockIdx.x; s < nseg; s += gridDim.x) {
    const int seg = (int)(s % segs);
    const long long row = s / segs;
    const int y = (int)(row % g.n), z = (int)((row / g.n) % g.n), b = (int)(row / ((long long)g.n * g.n));
    const int x0 = seg * 32;
    __syncthreads();  // the previous segment's reads are done
    for (int i = threadIdx.x; i < 32 * NC; i += blockDim.x) {
      const int xi = i / NC, o = i % NC, x = x0 + xi;
      const float v = x < g.n ? G[dense_index(b, z, y, x, g.n) * NC + o] : 0.f;
      bacc += v;
      Gt[o][xi] = __float2bfloat16_rn(v);
    }
    for (int i = threadIdx.x; i < 9 * 34 * NC; i += blockDim.x) {
      const int c = i % NC, xi = (i / NC) % 34, r = i / (NC * 34);
      const int zz = z + r / 3 - 1, yy = y + r % 3 - 1, xx = x0 + xi - 1;
      At[r][c][xi] = inside(zz, yy, xx, g.n) ? act[dense_index(b, zz, yy, xx, g.n) * NC + c] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int t = warp + 8 * j;
      if (t >= 27) break;
      const int r = t / 3, dx = t % 3;  // (dz, dy) row of the tile and x offset + 1
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const int k0 = ks * 16 + 2 * t4;
        unsigned a[4];
        a[0] = *(const unsigned *)&Gt[gq][k0];
        a[1] = *(const unsigned *)&Gt[gq + 8][k0];
        a[2] = *(const unsigned *)&Gt[gq][k0 + 8];
        a[3] = *(const unsigned *)&Gt[gq + 8][k0 + 8];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          const __nv_bfloat16 *src = &At[r][nt * 8 + gq][k0 + dx];
          const unsigned short s0 = __bfloat16_as_ushort(src[0]), s1 = __bfloat16_as_ushort(src[1]);
          const unsigned short s8 = __bfloat16_as_ushort(src[8]), s9 = __bfloat16_as_ushort(src[9]);
          const unsigned bb[2] = {(unsigned)s0 | ((unsigned)s1 << 16), (unsigned)s8 | ((unsigned)s9 << 16)};
          mma_bf16(acc[j][nt], a, bb);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int t = warp + 8 * j;
    if (t >= 27) break;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int o = gq + 8 * h, c = nt * 8 + 2 * t4;
        atomicAdd(dW + (o * 27 + t) * NC + c, acc[j][nt][2 * h]);
        atomicAdd(dW + (o * 27 + t) * NC + c + 1, acc[j][nt][2 * h + 1]);
      }
  }
  atomicAdd(db + (threadIdx.x % NC), bacc);
}

__device__ __forceinline__ bool is_bias(int i) {
  return (i >= kNetB1 && i < kNetB1 + NC) || (i >= kNetB2 && i < kNetB2 + NC) || i == kNetB3;
}

// Adam (Kingma & Ba, 2015) with bias-corrected moments; c1 = 1/(1-b1^k), c2 = 1/(1-b2^k)
__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ gr, float lr, float b1, float b2, float eps, float c1, float c2,
                            int train_bias) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kNetParams; i += gridDim.x * blockDim.x) {
    if (!train_bias && is_bias(i)) continue;
    const float gg = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * gg, vi = b2 * v[i] + (1.f - b2) * gg * gg;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// BF16 copies of W2: forward wf[t][o][c] = W2[o][t][c]; for the input gradient the
// transposed, tap-flipped wt[t][c][o] = W2[o][26 - t][c] (26 - t negates the offset)
__global__ void pack_w2_kernel(const float *__restrict__ prm, __nv_bfloat16 *__restrict__ wf,
                               __nv_bfloat16 *__restrict__ wt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 27 * NC * NC; i += gridDim.x * blockDim.x) {
    const int k = i % NC, j = (i / NC) % NC, t = i / (NC * NC);
    wf[i] = __float2bfloat16_rn(prm[kNetW2 + (j * 27 + t) * NC + k]);
    if (wt) wt[i] = __float2bfloat16_rn(prm[kNetW2 + (k * 27 + (26 - t)) * NC + j]);
  }
}

// ---------------------------------------------------------------- synthetic training pairs
__host__ __device__ __forceinline__ float kappa_of(unsigned long long seed, float klo, float khi, int b) {
  return klo + (khi - klo) * (float)uniform01(seed ^ 0x6b617070ULL, (unsigned long long)b);
}

__global__ void sample_kappa_kernel(int batch, unsigned long long seed, float klo, float khi, float *kappa) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch) kappa[b] = kappa_of(seed, klo, khi, b);
}

__global__ void sample_noise_kernel(long long npts, unsigned long long seed, float *__restrict__ t) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x)
    t[p] = (float)(2.0 * uniform01(seed, (unsigned long long)p) - 1.0);
}

// one colour of a Gauss-Seidel sweep of Ahat t = 0: t = kappa * (sum of neighbours) at
// points with (x + y + z) % 2 == parity (0-based; parity 1 = red, the 1-based even points)
__global__ void sample_gs_kernel(NetGrid g, const float *__restrict__ kappa, int parity, float *__restrict__ t) {
  const long long npts = (long long)g.batch * g.n * g.n * g.n;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x) {
    int b, z, y, x;
    split_point(p, g.n, b, z, y, x);
    if (((x + y + z) & 1) != parity) continue;
    t[p] = kappa[b] * nb6(t, b, z, y, x, g.n);
  }
}

__global__ void sample_ahat_kernel(NetGrid g, const float *__restrict__ kappa, const float *__restrict__ t,
                                   float *__restrict__ x) {
  const long long npts = (long long)g.batch * g.n * g.n * g.n;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x) {
    int b, z, y, xx;
    split_point(p, g.n, b, z, y, xx);
    x[p] = t[p] - kappa[b] * nb6(t, b, z, y, xx, g.n);
  }
}

// FP64 uniform noise in [-1, 1] (dense), the start of the multigrid-shaped samples
__global__ void sample_noise64_kernel(long long npts, unsigned long long seed, double *__restrict__ u) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x)
    u[p] = 2.0 * uniform01(seed, (unsigned long long)p) - 1.0;
}

// max |u| of every grid b of a dense batch into out[b] (bit pattern of the double)
__global__ void grid_maxabs_kernel(NetGrid g, const double *__restrict__ u, unsigned long long *__restrict__ out) {
  const long long npts = (long long)g.batch * g.slab;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x) {
    const double m = fabs(u[p]);
    // a warp may straddle two grids: reduce per lane only
    atomicMax(out + p / g.slab, (unsigned long long)__double_as_longlong(m));
  }
}

// t = u / max_b |u| (FP32), grids with max 0 stay 0
__global__ void normalise_kernel(NetGrid g, const double *__restrict__ u, const unsigned long long *__restrict__ mx,
                                 float *__restrict__ t) {
  const long long npts = (long long)g.batch * g.slab;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x) {
    const double m = __longlong_as_double((long long)mx[p / g.slab]);
    t[p] = m > 0.0 ? (float)(u[p] / m) : 0.f;
  }
}

// ---------------------------------------------------------------- multigrid level helpers
// padded level layout (pitch n + 1, no pad rows in y or z); neighbours outside the
// grid are zero
template <typename T>
__device__ __forceinline__ T lvl_nb6(const T *__restrict__ e, const Grid &g, long long i, int z, int y, int x) {
  T s = 0;
  if (x > 0) s += e[i - 1];
  if (x < g.n - 1) s += e[i + 1];
  if (y > 0) s += e[i - g.pitch];
  if (y < g.n - 1) s += e[i + g.pitch];
  if (z > 0) s += e[i - (long long)g.n * g.pitch];
  if (z < g.n - 1) s += e[i + (long long)g.n * g.pitch];
  return s;
}

// x = D^-1 (f - (I - c Lap) e) = f / D - e + kappa * (sum of neighbours of e)
template <typename T>
__global__ void net_resid_kernel(Grid g, double c, const T *__restrict__ e, const T *__restrict__ f, int batch,
                                 float *__restrict__ xout) {
  const double cih2 = c * g.ih2, D = 1.0 + 6.0 * cih2;
  const T iD = (T)(1.0 / D), kap = (T)(cih2 / D);
  const long long npts = (long long)batch * g.n * g.n * g.n;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npts; p += (long long)gridDim.x * blockDim.x) {
    int b, z, y, x;
    split_point(p, g.n, b, z, y, x);
    const long long i = b * g.slab + ((long long)z * g.n + y) * g.pitch + x;
    xout[i] = (float)(f[i] * iD - e[i] + kap * lvl_nb6(e, g, i, z, y, x));
  }
}

template <typename T>
__global__ void net_noise_kernel(Grid g, T *__restrict__ e, int batch, unsigned long long seed) {
  const long long tot = (long long)batch * g.slab;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.pitch);
    e[i] = x < g.n ? (T)(2.0 * uniform01(seed, (unsigned long long)i) - 1.0) : (T)0;
  }
}

template <typename T>
__global__ void net_maxabs_kernel(Grid g, const T *__restrict__ e, int batch, unsigned long long *out) {
  const long long tot = (long long)batch * g.slab;
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x)
    if ((int)(i % g.pitch) < g.n) m = fmax(m, fabs((double)e[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  // non-negative doubles order like their bit patterns
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// CTAs of the tiled 16 -> 16 layer: at most 4 per SM (48 KB of shared memory each), each
// walking several tiles so that the weights are staged once per CTA
int l2_tile_blocks(const NetGrid &g) {
  const long long tiles = (long long)g.batch * ((g.n + L2X - 1) / L2X) * ((g.n + L2Y - 1) / L2Y) *
                          ((g.n + L2Z - 1) / L2Z);
  const long long b = tiles < 152 * 4 * 4 ? tiles : 152 * 4 * 4;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t net_hidden(const Launch &L, const NetGrid &g, const float *x, const float *prm, const NetScratch &s) {
  const Grid gg = cube(g.n);
  const long long npts = (long long)g.batch * g.n * g.n * g.n;
  {
    Scope sc(L, K_NET_L1, gg, g.batch, 1);
    l1_fwd_kernel<<<grid_blocks(npts, 256), 256, 0, L.stream>>>(g, x, prm, s.a1);
    cudaError_t e = sc.done();
    if (e != cudaSuccess) return e;
  }
  Scope sc(L, K_NET_L2, gg, g.batch, 1);
  l2_tile_kernel<0><<<l2_tile_blocks(g), 256, 0, L.stream>>>(g, s.a1, s.w2f, prm + kNetB2, nullptr, s.a2, nullptr);
  return sc.done();
}

}  // namespace

// ---------------------------------------------------------------- scratch

size_t net_train_bytes(int batch, int n) {
  const size_t npts = (size_t)batch * n * n * n;
  return 3 * al256(npts * NC * 2) + 2 * al256(npts * NC * 4) + 5 * al256(npts * 4) + al256((size_t)batch * 4) +
         2 * al256(27 * NC * NC * 2);
}

NetScratch net_train_carve(void *base, int batch, int n) {
  const size_t npts = (size_t)batch * n * n * n;
  char *p = (char *)base;
  NetScratch s;
  auto take = [&](size_t bytes) { char *r = p; p += al256(bytes); return (void *)r; };
  s.a1 = (__nv_bfloat16 *)take(npts * NC * 2);
  s.a2 = (__nv_bfloat16 *)take(npts * NC * 2);
  s.gz2b = (__nv_bfloat16 *)take(npts * NC * 2);
  s.gz2 = (float *)take(npts * NC * 4);
  s.gz1 = (float *)take(npts * NC * 4);
  s.y = (float *)take(npts * 4);
  s.x = (float *)take(npts * 4);  // y - t
  s.w = (float *)take(npts * 4);
  s.gy = (float *)take(npts * 4);
  s.tmp = (float *)take(npts * 4);
  s.kappa = (float *)take((size_t)batch * 4);
  s.w2f = (__nv_bfloat16 *)take(27 * NC * NC * 2);
  s.w2t = (__nv_bfloat16 *)take(27 * NC * NC * 2);
  return s;
}

size_t net_infer_bytes(int batch, const Grid &g) {
  const size_t npts = (size_t)batch * g.n * g.n * g.n;
  return 2 * al256(npts * NC * 2) + al256((size_t)batch * g.slab * 4) + al256(27 * NC * NC * 2);
}

NetScratch net_infer_carve(void *base, int batch, const Grid &g) {
  const size_t npts = (size_t)batch * g.n * g.n * g.n;
  char *p = (char *)base;
  NetScratch s;
  auto take = [&](size_t bytes) { char *r = p; p += al256(bytes); return (void *)r; };
  s.a1 = (__nv_bfloat16 *)take(npts * NC * 2);
  s.a2 = (__nv_bfloat16 *)take(npts * NC * 2);
  s.x = (float *)take((size_t)batch * g.slab * 4);
  s.w2f = (__nv_bfloat16 *)take(27 * NC * NC * 2);
  return s;
}

// ---------------------------------------------------------------- host helpers

float net_sample_kappa(unsigned long long seed, float klo, float khi, int b) { return kappa_of(seed, klo, khi, b); }

int net_sample_vcycles(unsigned long long seed, int vmax, int b) {
  const int k = (int)(uniform01(seed ^ 0x76637963ULL, (unsigned long long)b) * (vmax + 1));
  return k > vmax ? vmax : k;
}

void net_init_params(float *prm, unsigned long long seed) {
  unsigned long long k = 0;
  auto normal = [&]() {  // Box-Muller on two counter-based uniforms
    const double u1 = 1.0 - uniform01(seed, k++), u2 = uniform01(seed, k++);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  };
  for (int i = 0; i < kNetParams; ++i) prm[i] = 0.f;
  for (int i = 0; i < NC * 27; ++i) prm[kNetW1 + i] = (float)(normal() * std::sqrt(2.0 / 27));
  for (int i = 0; i < NC * 27 * NC; ++i) prm[kNetW2 + i] = (float)(normal() * std::sqrt(2.0 / (27 * NC)));
  for (int i = 0; i < 27 * NC; ++i) prm[kNetW3 + i] = (float)(normal() * std::sqrt(1.0 / (27 * NC)));
}

// ---------------------------------------------------------------- launchers

cudaError_t k_net_pack(const Launch &L, const float *prm, const NetScratch &s) {
  pack_w2_kernel<<<27, 256, 0, L.stream>>>(prm, s.w2f, s.w2t);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

cudaError_t k_net_forward(const Launch &L, const NetGrid &g, const float *x, const float *prm, const NetScratch &s,
                          float *y) {
  cudaError_t e = net_hidden(L, g, x, prm, s);
  if (e != cudaSuccess) return e;
  const long long npts = (long long)g.batch * g.n * g.n * g.n;
  Scope sc(L, K_NET_L3, cube(g.n), g.batch, 1);
  l3_fwd_kernel<float, false><<<grid_blocks(npts, 256), 256, 0, L.stream>>>(g, s.a2, prm, y);
  return sc.done();
}

// g must be the dense layout (pitch n, slab n^3)
cudaError_t k_net_grads(const Launch &L, const NetGrid &g, const float *x, const float *t, const float *kappa,
                        int power, const float *prm, float *grad, const NetScratch &s, double *loss) {
  const Grid gg = cube(g.n);
  const long long npts = (long long)g.batch * g.n * g.n * g.n;
  const int nb = grid_blocks(npts, 256), wb = 152 * 2;
  cudaError_t e = k_net_forward(L, g, x, prm, s, s.y);
  if (e != cudaSuccess) return e;
#define PMG_NET_STEP(kid, launch)      \
  do {                                 \
    Scope sc_(L, kid, gg, g.batch, 1); \
    launch;                            \
    cudaError_t e_ = sc_.done();       \
    if (e_ != cudaSuccess) return e_;  \
  } while (0)
  // d = y - t; w = Ahat^power d; loss; gy = Ahat^power w / count (Ahat is symmetric)
  PMG_NET_STEP(K_NET_LOSS, (net_diff_kernel<<<nb, 256, 0, L.stream>>>(npts, s.y, t, s.x)));
  const float *cur = s.x;
  for (int i = 0; i < power; ++i) {
    float *out = cur == s.w ? s.tmp : s.w;
    PMG_NET_STEP(K_NET_LOSS, (net_ahat_kernel<<<nb, 256, 0, L.stream>>>(g, cur, kappa, 1.f, out)));
    cur = out;
  }
  PMG_NET_STEP(K_NET_LOSS, (net_sqloss_kernel<<<nb, 256, 0, L.stream>>>(npts, cur, 1.0 / npts, loss)));
  const float inv = (float)(1.0 / npts);
  if (power == 0) PMG_NET_STEP(K_NET_LOSS, (net_scale_kernel<<<nb, 256, 0, L.stream>>>(npts, cur, inv, s.gy)));
  for (int i = 0; i < power; ++i) {
    const bool last = i == power - 1;
    float *out = last ? s.gy : (cur == s.w ? s.tmp : s.w);
    PMG_NET_STEP(K_NET_LOSS, (net_ahat_kernel<<<nb, 256, 0, L.stream>>>(g, cur, kappa, last ? inv : 1.f, out)));
    cur = out;
  }
  PMG_NET_STEP(K_NET_WGRAD,
               (wgrad_kernel<1, NC, __nv_bfloat16><<<wb, 256, 0, L.stream>>>(g, s.gy, s.a2, grad + kNetW3,
                                                                            grad + kNetB3)));
  PMG_NET_STEP(K_NET_L3BWD, (l3_bwd_data_kernel<<<nb, 256, 0, L.stream>>>(g, s.gy, s.a2, prm, s.gz2, s.gz2b)));
  PMG_NET_STEP(K_NET_WGRAD,
               (wgrad_mma_kernel<<<wb, 256, 0, L.stream>>>(g, s.gz2, s.a1, grad + kNetW2, grad + kNetB2)));
  PMG_NET_STEP(K_NET_L2BWD, (l2_tile_kernel<1><<<l2_tile_blocks(g), 256, 0, L.stream>>>(g, s.gz2b, s.w2t, nullptr,
                                                                                       s.a1, nullptr, s.gz1)));
  PMG_NET_STEP(K_NET_WGRAD, (wgrad_kernel<NC, 1, float><<<wb, 256, 0, L.stream>>>(g, s.gz1, x, grad + kNetW1,
                                                                                 grad + kNetB1)));
#undef PMG_NET_STEP
  return cudaSuccess;
}

cudaError_t k_net_adam(const Launch &L, float *prm, float *m, float *v, const float *grad, int step, float lr,
                       float b1, float b2, float eps, bool train_bias) {
  const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, step)));
  const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, step)));
  Scope sc(L, K_NET_ADAM, cube(3), 1, 1);
  adam_kernel<<<32, 256, 0, L.stream>>>(prm, m, v, grad, lr, b1, b2, eps, c1, c2, train_bias ? 1 : 0);
  return sc.done();
}

cudaError_t k_net_sample(const Launch &L, const NetGrid &g, unsigned long long seed, float klo, float khi, float *x,
                         float *t, float *kappa) {
  const long long npts = (long long)g.batch * g.n * g.n * g.n;
  const int nb = grid_blocks(npts, 256);
  Scope sc(L, K_NET_SAMPLE, cube(g.n), g.batch, 1);
  sample_kappa_kernel<<<(g.batch + 127) / 128, 128, 0, L.stream>>>(g.batch, seed, klo, khi, kappa);
  sample_noise_kernel<<<nb, 256, 0, L.stream>>>(npts, seed, t);
  sample_gs_kernel<<<nb, 256, 0, L.stream>>>(g, kappa, 1, t);  // red first
  sample_gs_kernel<<<nb, 256, 0, L.stream>>>(g, kappa, 0, t);
  sample_ahat_kernel<<<nb, 256, 0, L.stream>>>(g, kappa, t, x);
  if (L.counter) *L.counter += 4;  // Scope::done counts the fifth
  return sc.done();
}

cudaError_t k_net_sample_noise64(const Launch &L, const NetGrid &g, unsigned long long seed, double *u) {
  const long long npts = (long long)g.batch * g.slab;
  sample_noise64_kernel<<<grid_blocks(npts, 256), 256, 0, L.stream>>>(npts, seed, u);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

// a -= b over n FP64 values (the initial error u* - u0 of a sub-step solve)
__global__ void sub64_kernel(long long n, double *__restrict__ a, const double *__restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] -= b[i];
}

cudaError_t k_net_sub64(const Launch &L, const NetGrid &g, double *a, const double *b) {
  const long long npts = (long long)g.batch * g.slab;
  Scope sc(L, K_NET_SAMPLE, cube(g.n), g.batch, 0);
  sub64_kernel<<<grid_blocks(npts, 256), 256, 0, L.stream>>>(npts, a, b);
  return sc.done();
}

cudaError_t k_net_sample_finish(const Launch &L, const NetGrid &g, const double *u, unsigned long long *mx,
                                float *x, float *t, const float *kappa) {
  const long long npts = (long long)g.batch * g.slab;
  const int nb = grid_blocks(npts, 256);
  Scope sc(L, K_NET_SAMPLE, cube(g.n), g.batch, 1);
  cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * g.batch, L.stream);
  grid_maxabs_kernel<<<nb, 256, 0, L.stream>>>(g, u, mx);
  normalise_kernel<<<nb, 256, 0, L.stream>>>(g, u, mx, t);
  sample_gs_kernel<<<nb, 256, 0, L.stream>>>(g, kappa, 1, t);  // red first
  sample_gs_kernel<<<nb, 256, 0, L.stream>>>(g, kappa, 0, t);
  sample_ahat_kernel<<<nb, 256, 0, L.stream>>>(g, kappa, t, x);
  if (L.counter) *L.counter += 4;
  return sc.done();
}

cudaError_t k_net_correct(const Launch &L, const Grid &g, double c, Prec pr, void *e, const void *f, int batch,
                          const float *prm, const NetScratch &s) {
  const long long npts = (long long)batch * g.n * g.n * g.n;
  const int nb = grid_blocks(npts, 256);
  {
    Scope sc(L, K_NET_RESID, g, batch, pr);
    if (pr == F32)
      net_resid_kernel<float><<<nb, 256, 0, L.stream>>>(g, c, (const float *)e, (const float *)f, batch, s.x);
    else
      net_resid_kernel<double><<<nb, 256, 0, L.stream>>>(g, c, (const double *)e, (const double *)f, batch, s.x);
    cudaError_t err = sc.done();
    if (err != cudaSuccess) return err;
  }
  const NetGrid ng{batch, g.n, g.pitch, g.slab};
  cudaError_t err = net_hidden(L, ng, s.x, prm, s);
  if (err != cudaSuccess) return err;
  Scope sc(L, K_NET_L3, g, batch, pr);
  if (pr == F32) l3_fwd_kernel<float, true><<<nb, 256, 0, L.stream>>>(ng, s.a2, prm, (float *)e);
  else l3_fwd_kernel<double, true><<<nb, 256, 0, L.stream>>>(ng, s.a2, prm, (double *)e);
  return sc.done();
}

cudaError_t k_net_noise(const Launch &L, const Grid &g, Prec pr, void *e, int batch, unsigned long long seed) {
  const int nb = grid_blocks((long long)batch * g.slab, 256);
  if (pr == F32) net_noise_kernel<float><<<nb, 256, 0, L.stream>>>(g, (float *)e, batch, seed);
  else net_noise_kernel<double><<<nb, 256, 0, L.stream>>>(g, (double *)e, batch, seed);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

cudaError_t k_net_maxabs(const Launch &L, const Grid &g, Prec pr, const void *e, int batch, unsigned long long *out) {
  const int nb = grid_blocks((long long)batch * g.slab, 256);
  if (pr == F32) net_maxabs_kernel<float><<<nb, 256, 0, L.stream>>>(g, (const float *)e, batch, out);
  else net_maxabs_kernel<double><<<nb, 256, 0, L.stream>>>(g, (const double *)e, batch, out);
  if (L.counter) ++*L.counter;
  return cudaGetLastError();
}

}  // namespace pmg
