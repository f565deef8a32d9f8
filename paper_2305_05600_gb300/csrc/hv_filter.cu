// Learned moment filter (x-z layout): a residual 3x3 convolutional network
// 4 -> 16 -> 16 -> 4 (ReLU between layers, periodic padding) applied to the
// deposited half-step moments (n, Jx, Jy, Jz), with the binomial smoothing
// as a gated fallback:
//   x = m / s,  h1 = bf16(relu(conv(bf16(x)))),  h2 = bf16(relu(conv(h1))),
//   f = conv(h2),  y = m + s f   unless n < nmin or |s_n f_n| > rmax max(n, n_f),
//   where y is one (1/4, 1/2, 1/4) pass per axis of m.
// The paper smooths noisy moments with binomial passes (Sec. 2.2); the
// network is an addition that the smoothing backs up.
//
// Each block filters one 16x16 tile.  The three convolutions are implicit
// GEMMs on the tensor cores (mma.sync m16n8k16, bf16 x bf16 -> fp32): rows are
// the pixels of a layer's output region (the tile plus a halo shrinking from
// 2 to 0), columns the output channels, and the reduction runs over
// (tap, input channel).  Activations stay in shared memory as bf16.
#include <vector>

#include "hv_internal.cuh"

namespace hv {

namespace {

constexpr int kFT = 16;                       // tile extent (x and z)
constexpr int kR0 = kFT + 6, kR1 = kFT + 4;   // input region (halo 3), h1 region (halo 2)
constexpr int kR2 = kFT + 2;                  // h2 region (halo 1)
constexpr int kN0 = kR0 * kR0, kN1 = kR1 * kR1, kN2 = kR2 * kR2, kN3 = kFT * kFT;
constexpr int kK1 = 48, kK2 = 144, kK3 = 144;  // GEMM depths (layer 1 padded from 36)
constexpr int kHS = 24;                        // bf16 per pixel row of h1/h2 (16 + pad)
constexpr int kWOff2 = 16 * kK1, kWOff3 = kWOff2 + 16 * kK2, kWTotal = kWOff3 + 8 * kK3;
constexpr int kThreads = 128;

struct Smem {
  __nv_bfloat16 x[kN0][4];            // bf16(m / s) on the input region
  __nv_bfloat16 h1[kN1][kHS];
  __nv_bfloat16 h2[kN2][kHS];
  __nv_bfloat16 w[kWTotal];
  float bias[40];
  float4 raw[kR2 * kR2];              // raw moments on the tile + 1 (fallback, residual)
  float f[kN3][4];                    // network output on the tile
};

__device__ __forceinline__ void mma16816(float *d, const uint32_t *a, const uint32_t *b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p) {
  return *reinterpret_cast<const uint32_t *>(p);
}

// One convolution layer as an implicit GEMM.  Output region: RO x RO pixels
// (row-major), input region RI = RO + 2.  CIN channels per input pixel
// (4 for layer 1, laid out [pixel][4]; 16 otherwise, [pixel][kHS]).  NT
// n-tiles of 8 output channels.  The epilogue functor receives (pixel,
// channel, value) for channels < COUT.
template <int CIN, int RO, int K, int NT, int COUT, class In, class Epi>
__device__ __forceinline__ void conv_layer(const In &in_at, const __nv_bfloat16 *W,
                                           const float *bias, Epi epi) {
  constexpr int RI = RO + 2;
  constexpr int NPIX = RO * RO;
  constexpr int MT = (NPIX + 15) / 16;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  for (int mt = warp; mt < MT; mt += kThreads / 32) {
    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    // the two pixel rows this thread feeds (clamped: padded rows are not stored)
    const int p0 = min(mt * 16 + gid, NPIX - 1), p1 = min(mt * 16 + gid + 8, NPIX - 1);
    const int x0 = p0 % RO, z0 = p0 / RO, x1 = p1 % RO, z1 = p1 / RO;
#pragma unroll
    for (int ks = 0; ks < K / 16; ++ks) {
      uint32_t a[4];
      if (CIN == 4) {
        // k = tap * 4 + ci; this thread's columns tig*2+{0,1} and +8
        const int tapA = ks * 4 + (tig >> 1), tapB = tapA + 2, ci = (tig & 1) * 2;
        auto ldx = [&](int x, int z, int tap) -> uint32_t {
          if (tap >= 9) return 0u;
          const int da = tap % 3, db = tap / 3;  // input region is shifted by +1
          return ld32(in_at(x + da, z + db) + ci);
        };
        a[0] = ldx(x0, z0, tapA);
        a[1] = ldx(x1, z1, tapA);
        a[2] = ldx(x0, z0, tapB);
        a[3] = ldx(x1, z1, tapB);
      } else {
        // k = tap * 16 + ci: one tap per k-step, channels tig*2+{0,1} and +8
        const int tap = ks, da = tap % 3, db = tap / 3, ci = tig * 2;
        const __nv_bfloat16 *r0 = in_at(x0 + da, z0 + db), *r1 = in_at(x1 + da, z1 + db);
        a[0] = ld32(r0 + ci);
        a[1] = ld32(r1 + ci);
        a[2] = ld32(r0 + ci + 8);
        a[3] = ld32(r1 + ci + 8);
      }
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        // B is stored [n][K]: rows k = tig*2+{0,1} (+8) of column n*8+gid
        const __nv_bfloat16 *wc = W + (n * 8 + gid) * K + ks * 16 + tig * 2;
        uint32_t b[2] = {ld32(wc), ld32(wc + 8)};
        mma16816(acc[n], a, b);
      }
    }
    // epilogue: rows gid, gid+8; columns tig*2+{0,1} of each n-tile
#pragma unroll
    for (int n = 0; n < NT; ++n)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int p = mt * 16 + gid + 8 * h;
        if (p >= NPIX) continue;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int co = n * 8 + tig * 2 + j;
          if (co < COUT) epi(p, co, acc[n][2 * h + j] + bias[co]);
        }
      }
  }
  (void)RI;
}

__device__ __forceinline__ int wrapn(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

__global__ void __launch_bounds__(kThreads) filter_kernel(Geom g, FilterParams fp, float nfloor,
                                                          const float4 *m, float4 *y) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Smem &S = *reinterpret_cast<Smem *>(smraw);
  const int ntx = (g.nx + kFT - 1) / kFT;
  const int x0 = (blockIdx.x % ntx) * kFT, z0 = (blockIdx.x / ntx) * kFT;
  const float is0 = 1.f / fp.scale[0], is1 = 1.f / fp.scale[1], is2 = 1.f / fp.scale[2],
              is3 = 1.f / fp.scale[3];
  // weights and biases
  for (int i = threadIdx.x; i < kWTotal / 2; i += kThreads)
    reinterpret_cast<uint32_t *>(S.w)[i] = reinterpret_cast<const uint32_t *>(fp.w)[i];
  for (int i = threadIdx.x; i < 40; i += kThreads) S.bias[i] = fp.bias[i];
  // inputs: bf16(m / s) on the tile + 3, raw m on the tile + 1 (periodic)
  for (int t = threadIdx.x; t < kN0; t += kThreads) {
    const int rx = t % kR0 - 3, rz = t / kR0 - 3;
    const int gi = wrapn(x0 + rx, g.nx), gk = wrapn(z0 + rz, g.nz);
    const float4 v = m[gi + g.nx * gk];
    S.x[t][0] = __float2bfloat16_rn(v.x * is0);
    S.x[t][1] = __float2bfloat16_rn(v.y * is1);
    S.x[t][2] = __float2bfloat16_rn(v.z * is2);
    S.x[t][3] = __float2bfloat16_rn(v.w * is3);
    if (rx >= -1 && rx <= kFT && rz >= -1 && rz <= kFT) S.raw[(rx + 1) + (rz + 1) * kR2] = v;
  }
  __syncthreads();
  // layer 1: 4 -> 16 on the h1 region (tile + 2)
  conv_layer<4, kR1, kK1, 2, 16>(
      [&](int x, int z) { return &S.x[x + z * kR0][0]; }, S.w, S.bias,
      [&](int p, int co, float v) { S.h1[p][co] = __float2bfloat16_rn(fmaxf(v, 0.f)); });
  __syncthreads();
  // layer 2: 16 -> 16 on the h2 region (tile + 1)
  conv_layer<16, kR2, kK2, 2, 16>(
      [&](int x, int z) { return &S.h1[x + z * kR1][0]; }, S.w + kWOff2, S.bias + 16,
      [&](int p, int co, float v) { S.h2[p][co] = __float2bfloat16_rn(fmaxf(v, 0.f)); });
  __syncthreads();
  // layer 3: 16 -> 4 on the tile
  conv_layer<16, kFT, kK3, 1, 4>(
      [&](int x, int z) { return &S.h2[x + z * kR2][0]; }, S.w + kWOff3, S.bias + 32,
      [&](int p, int co, float v) { S.f[p][co] = v; });
  __syncthreads();
  // residual, gate and binomial fallback
  for (int p = threadIdx.x; p < kN3; p += kThreads) {
    const int tx = p % kFT, tz = p / kFT;
    const int gx = x0 + tx, gz = z0 + tz;
    if (gx >= g.nx || gz >= g.nz) continue;
    const float4 c = S.raw[(tx + 1) + (tz + 1) * kR2];
    const float rn = fabsf(fp.scale[0] * S.f[p][0]);
    const bool fallback = c.x < fp.nmin || rn > fp.rmax * fmaxf(c.x, nfloor);
    float4 out;
    if (fallback) {
      const float w1[3] = {0.25f, 0.5f, 0.25f};
      out = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          const float wgt = w1[a] * w1[b];
          const float4 q = S.raw[(tx + a) + (tz + b) * kR2];
          out.x = fmaf(wgt, q.x, out.x);
          out.y = fmaf(wgt, q.y, out.y);
          out.z = fmaf(wgt, q.z, out.z);
          out.w = fmaf(wgt, q.w, out.w);
        }
    } else {
      out = make_float4(c.x + fp.scale[0] * S.f[p][0], c.y + fp.scale[1] * S.f[p][1],
                        c.z + fp.scale[2] * S.f[p][2], c.w + fp.scale[3] * S.f[p][3]);
    }
    y[gx + g.nx * gz] = out;
  }
}


// ----------------------------------------------------------------------------
// Training: loss = mean over cells, channels and batch of (x + f(x) - t)^2,
// x = m / s, t = target / s.  One block per (16x16 tile, batch item) runs the
// forward pass on the tile plus a halo of 2 (so that the backward pass has
// the output gradient on the halo it needs), then the backward pass:
//   dF = 2 (x + f - t) / N                     on tile + 2
//   dH2 = conv^T(dF, W3) masked by h2 > 0      on tile + 1  (tensor cores)
//   dH1 = conv^T(dH2, W2) masked by h1 > 0     on the tile  (tensor cores)
// and adds the weight and bias gradients of its tile's output pixels
// (FP32 CUDA cores) into the global gradient.  conv^T is the correlation with
// the kernel flipped and its channel axes swapped.
// ----------------------------------------------------------------------------
constexpr int kT5 = kFT + 10, kT4 = kFT + 8, kT3 = kFT + 6, kT2 = kFT + 4, kT1 = kFT + 2;
constexpr int kWT3 = 16 * kK1;            // W3 transposed: [16 ci][48 = tap*4 + co]
constexpr int kWT2 = 16 * kK2;            // W2 transposed: [16 ci][144 = tap*16 + co]

struct TrainSmem {
  __nv_bfloat16 x[kT5 * kT5][4];          // bf16(m / s) on tile + 5
  __nv_bfloat16 h1[kT4 * kT4][kHS];       // on tile + 4
  __nv_bfloat16 h2[kT3 * kT3][kHS];       // on tile + 3
  __nv_bfloat16 dfb[kT2 * kT2][4];        // bf16 dF on tile + 2
  __nv_bfloat16 dh2[kT1 * kT1][kHS];      // masked dH2 on tile + 1
  float df[kT2 * kT2][4];                 // fp32 dF
  float dh1[kN3][16];                     // masked dH1 on the tile
  float xs[kT2 * kT2][4];                 // m / s on tile + 2 (residual)
  float ts[kT2 * kT2][4];                 // target / s on tile + 2
  __nv_bfloat16 w[kWTotal];
  __nv_bfloat16 wt3[kWT3];
  __nv_bfloat16 wt2[kWT2];
  float bias[40];
  float zero[16];                         // no bias in the backward convolutions
  double loss;
};

__global__ void __launch_bounds__(kThreads) filter_grad_kernel(Geom g, FilterParams fp,
                                                               const __nv_bfloat16 *wt,
                                                               const float4 *m, const float4 *tg,
                                                               float inv_count, float *grad,
                                                               double *loss) {
  extern __shared__ __align__(16) unsigned char smraw[];
  TrainSmem &S = *reinterpret_cast<TrainSmem *>(smraw);
  const int ntx = (g.nx + kFT - 1) / kFT;
  const int x0 = (blockIdx.x % ntx) * kFT, z0 = (blockIdx.x / ntx) * kFT;
  const size_t boff = (size_t)blockIdx.y * g.ncell;
  const float4 *mb = m + boff, *tb = tg + boff;
  const float is[4] = {1.f / fp.scale[0], 1.f / fp.scale[1], 1.f / fp.scale[2],
                       1.f / fp.scale[3]};
  for (int i = threadIdx.x; i < kWTotal / 2; i += kThreads)
    reinterpret_cast<uint32_t *>(S.w)[i] = reinterpret_cast<const uint32_t *>(fp.w)[i];
  for (int i = threadIdx.x; i < (kWT3 + kWT2) / 2; i += kThreads) {
    const uint32_t v = reinterpret_cast<const uint32_t *>(wt)[i];
    if (i < kWT3 / 2) reinterpret_cast<uint32_t *>(S.wt3)[i] = v;
    else reinterpret_cast<uint32_t *>(S.wt2)[i - kWT3 / 2] = v;
  }
  for (int i = threadIdx.x; i < 40; i += kThreads) S.bias[i] = fp.bias[i];
  for (int i = threadIdx.x; i < 16; i += kThreads) S.zero[i] = 0.f;
  if (threadIdx.x == 0) S.loss = 0.0;
  for (int t = threadIdx.x; t < kT5 * kT5; t += kThreads) {
    const int rx = t % kT5 - 5, rz = t / kT5 - 5;
    const int gi = wrapn(x0 + rx, g.nx), gk = wrapn(z0 + rz, g.nz);
    const float4 v = mb[gi + g.nx * gk];
    const float xv[4] = {v.x * is[0], v.y * is[1], v.z * is[2], v.w * is[3]};
#pragma unroll
    for (int c = 0; c < 4; ++c) S.x[t][c] = __float2bfloat16_rn(xv[c]);
    if (rx >= -2 && rx < kFT + 2 && rz >= -2 && rz < kFT + 2) {
      const int q = (rx + 2) + (rz + 2) * kT2;
      const float4 u = tb[gi + g.nx * gk];
      const float tv[4] = {u.x * is[0], u.y * is[1], u.z * is[2], u.w * is[3]};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        S.xs[q][c] = xv[c];
        S.ts[q][c] = tv[c];
      }
    }
  }
  __syncthreads();
  // forward on the enlarged regions
  conv_layer<4, kT4, kK1, 2, 16>(
      [&](int x, int z) { return &S.x[x + z * kT5][0]; }, S.w, S.bias,
      [&](int p, int co, float v) { S.h1[p][co] = __float2bfloat16_rn(fmaxf(v, 0.f)); });
  __syncthreads();
  conv_layer<16, kT3, kK2, 2, 16>(
      [&](int x, int z) { return &S.h1[x + z * kT4][0]; }, S.w + kWOff2, S.bias + 16,
      [&](int p, int co, float v) { S.h2[p][co] = __float2bfloat16_rn(fmaxf(v, 0.f)); });
  __syncthreads();
  // f on tile + 2, then dF (only pixels inside the grid count)
  conv_layer<16, kT2, kK3, 1, 4>(
      [&](int x, int z) { return &S.h2[x + z * kT3][0]; }, S.w + kWOff3, S.bias + 32,
      [&](int p, int co, float v) {
        const float e = S.xs[p][co] + v - S.ts[p][co];
        S.df[p][co] = 2.f * e * inv_count;
        S.dfb[p][co] = __float2bfloat16_rn(2.f * e * inv_count);
        const int tx = p % kT2 - 2, tz = p / kT2 - 2;
        if (tx >= 0 && tx < kFT && tz >= 0 && tz < kFT && x0 + tx < g.nx && z0 + tz < g.nz)
          atomicAdd(&S.loss, (double)(e * e) * (double)inv_count);
      });
  __syncthreads();
  // dH2 on tile + 1: conv^T(dF, W3), masked by h2 > 0
  conv_layer<4, kT1, kK1, 2, 16>(
      [&](int x, int z) { return &S.dfb[x + z * kT2][0]; }, S.wt3, S.zero,
      [&](int p, int co, float v) {
        const int hx = p % kT1 + 2, hz = p / kT1 + 2;  // same point in the h2 region
        const float h = __bfloat162float(S.h2[hx + hz * kT3][co]);
        S.dh2[p][co] = __float2bfloat16_rn(h > 0.f ? v : 0.f);
      });
  __syncthreads();
  // dH1 on the tile: conv^T(dH2, W2), masked by h1 > 0
  conv_layer<16, kFT, kK2, 2, 16>(
      [&](int x, int z) { return &S.dh2[x + z * kT1][0]; }, S.wt2, S.zero,
      [&](int p, int co, float v) {
        const int hx = p % kFT + 4, hz = p / kFT + 4;
        const float h = __bfloat162float(S.h1[hx + hz * kT4][co]);
        S.dh1[p][co] = h > 0.f ? v : 0.f;
      });
  __syncthreads();
  // weight and bias gradients from the tile's pixels (inside the grid)
  const int vx = min(kFT, g.nx - x0), vz = min(kFT, g.nz - z0);
  for (int q = threadIdx.x; q < kFilterParams; q += kThreads) {
    float acc = 0.f;
    if (q < 576) {  // W1[o][c][tap]: dH1 x xb
      const int o = q / 36, c = (q / 9) % 4, tap = q % 9, da = tap % 3 - 1, db = tap / 3 - 1;
      for (int pz = 0; pz < vz; ++pz)
        for (int px = 0; px < vx; ++px)
          acc = fmaf(S.dh1[px + pz * kFT][o],
                     __bfloat162float(S.x[(px + 5 + da) + (pz + 5 + db) * kT5][c]), acc);
    } else if (q < 592) {  // b1
      const int o = q - 576;
      for (int pz = 0; pz < vz; ++pz)
        for (int px = 0; px < vx; ++px) acc += S.dh1[px + pz * kFT][o];
    } else if (q < 2896) {  // W2: dH2 x h1
      const int r = q - 592, o = r / 144, c = (r / 9) % 16, tap = r % 9, da = tap % 3 - 1,
                db = tap / 3 - 1;
      for (int pz = 0; pz < vz; ++pz)
        for (int px = 0; px < vx; ++px)
          acc = fmaf(__bfloat162float(S.dh2[(px + 1) + (pz + 1) * kT1][o]),
                     __bfloat162float(S.h1[(px + 4 + da) + (pz + 4 + db) * kT4][c]), acc);
    } else if (q < 2912) {  // b2
      const int o = q - 2896;
      for (int pz = 0; pz < vz; ++pz)
        for (int px = 0; px < vx; ++px)
          acc += __bfloat162float(S.dh2[(px + 1) + (pz + 1) * kT1][o]);
    } else if (q < 3488) {  // W3: dF x h2
      const int r = q - 2912, o = r / 144, c = (r / 9) % 16, tap = r % 9, da = tap % 3 - 1,
                db = tap / 3 - 1;
      for (int pz = 0; pz < vz; ++pz)
        for (int px = 0; px < vx; ++px)
          acc = fmaf(S.df[(px + 2) + (pz + 2) * kT2][o],
                     __bfloat162float(S.h2[(px + 3 + da) + (pz + 3 + db) * kT3][c]), acc);
    } else {  // b3
      const int o = q - 3488;
      for (int pz = 0; pz < vz; ++pz)
        for (int px = 0; px < vx; ++px) acc += S.df[(px + 2) + (pz + 2) * kT2][o];
    }
    atomicAdd(grad + q, acc);
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(loss, S.loss);
}

// Adam on the FP32 master parameters, then refresh the packed bf16 weights:
// forward layouts (as pack_filter) and the transposed, flipped layouts of
// W3 and W2 used by the backward pass.
__global__ void adam_kernel(float *P, float *grad, float *mom1, float *mom2, int t, float lr,
                            __nv_bfloat16 *w, float *bias, __nv_bfloat16 *wt) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kFilterParams;
       q += gridDim.x * blockDim.x) {
    const float gq = grad[q];
    const float m1 = b1 * mom1[q] + (1.f - b1) * gq;
    const float m2 = b2 * mom2[q] + (1.f - b2) * gq * gq;
    mom1[q] = m1;
    mom2[q] = m2;
    const float v = P[q] - lr * (m1 / c1) / (sqrtf(m2 / c2) + eps);
    P[q] = v;
    grad[q] = 0.f;
    const __nv_bfloat16 vb = __float2bfloat16_rn(v);
    if (q < 576) {
      const int o = q / 36, c = (q / 9) % 4, tap = q % 9;
      w[o * kK1 + tap * 4 + c] = vb;
    } else if (q < 592) {
      bias[q - 576] = v;
    } else if (q < 2896) {
      const int r = q - 592, o = r / 144, c = (r / 9) % 16, tap = r % 9;
      w[kWOff2 + o * kK2 + tap * 16 + c] = vb;
      wt[kWT3 + c * kK2 + (8 - tap) * 16 + o] = vb;  // W2^T flipped: [c][tap'*16 + o]
    } else if (q < 2912) {
      bias[16 + q - 2896] = v;
    } else if (q < 3488) {
      const int r = q - 2912, o = r / 144, c = (r / 9) % 16, tap = r % 9;
      w[kWOff3 + o * kK3 + tap * 16 + c] = vb;
      wt[c * kK1 + (8 - tap) * 4 + o] = vb;          // W3^T flipped: [c][tap'*4 + o]
    } else {
      bias[32 + q - 3488] = v;
    }
  }
}

}  // namespace

size_t filter_smem_bytes() { return sizeof(Smem); }

cudaError_t launch_filter(hv_ctx *c, const FilterParams &fp, const float4 *in, float4 *out) {
  static std::atomic<uint64_t> attr_set{0};
  cudaError_t e = set_smem_once(filter_kernel, sizeof(Smem), attr_set);
  if (e != cudaSuccess) return e;
  const int ntx = (c->g.nx + kFT - 1) / kFT, ntz = (c->g.nz + kFT - 1) / kFT;
  c->launches++;
  filter_kernel<<<ntx * ntz, kThreads, sizeof(Smem), c->stream>>>(c->g, fp, (float)c->p.n_floor,
                                                                   in, out);
  return cudaGetLastError();
}

// Pack float parameters (W1[16][4][3][3] b1 W2[16][16][3][3] b2 W3[4][16][3][3]
// b3) into the GEMM layouts: B matrices stored [n][K], k = tap * cin + ci,
// tap = 3 * (db + 1) + (da + 1).
void pack_filter(const float *P, std::vector<__nv_bfloat16> &w, std::vector<float> &bias) {
  static_assert(kFilterParams == 3492, "parameter count");
  w.assign(kWTotal, __float2bfloat16(0.f));
  bias.assign(40, 0.f);
  const float *W1 = P, *b1 = W1 + 576, *W2 = b1 + 16, *b2 = W2 + 2304, *W3 = b2 + 16,
              *b3 = W3 + 576;
  for (int o = 0; o < 16; ++o)
    for (int ci = 0; ci < 4; ++ci)
      for (int tap = 0; tap < 9; ++tap)
        w[o * kK1 + tap * 4 + ci] = __float2bfloat16(W1[(o * 4 + ci) * 9 + tap]);
  for (int o = 0; o < 16; ++o)
    for (int ci = 0; ci < 16; ++ci)
      for (int tap = 0; tap < 9; ++tap)
        w[kWOff2 + o * kK2 + tap * 16 + ci] = __float2bfloat16(W2[(o * 16 + ci) * 9 + tap]);
  for (int o = 0; o < 4; ++o)
    for (int ci = 0; ci < 16; ++ci)
      for (int tap = 0; tap < 9; ++tap)
        w[kWOff3 + o * kK3 + tap * 16 + ci] = __float2bfloat16(W3[(o * 16 + ci) * 9 + tap]);
  for (int i = 0; i < 16; ++i) bias[i] = b1[i];
  for (int i = 0; i < 16; ++i) bias[16 + i] = b2[i];
  for (int i = 0; i < 4; ++i) bias[32 + i] = b3[i];
}

int filter_weight_count() { return kWTotal; }

size_t filter_train_weight_count() { return (size_t)kWT3 + kWT2; }

// Transposed, flipped bf16 copies of W3 and W2 for the backward pass.
void pack_filter_transposed(const float *P, std::vector<__nv_bfloat16> &wt) {
  wt.assign(kWT3 + kWT2, __float2bfloat16(0.f));
  const float *W2 = P + 592, *W3 = P + 2912;
  for (int o = 0; o < 16; ++o)
    for (int c = 0; c < 16; ++c)
      for (int tap = 0; tap < 9; ++tap)
        wt[kWT3 + c * kK2 + (8 - tap) * 16 + o] = __float2bfloat16(W2[(o * 16 + c) * 9 + tap]);
  for (int o = 0; o < 4; ++o)
    for (int c = 0; c < 16; ++c)
      for (int tap = 0; tap < 9; ++tap)
        wt[c * kK1 + (8 - tap) * 4 + o] = __float2bfloat16(W3[(o * 16 + c) * 9 + tap]);
}

cudaError_t launch_filter_grad(hv_ctx *c, const FilterParams &fp, const __nv_bfloat16 *wt,
                               const float4 *m, const float4 *tg, int nbatch, float *grad,
                               double *loss) {
  static std::atomic<uint64_t> attr_set{0};
  cudaError_t e = set_smem_once(filter_grad_kernel, sizeof(TrainSmem), attr_set);
  if (e != cudaSuccess) return e;
  const int ntx = (c->g.nx + kFT - 1) / kFT, ntz = (c->g.nz + kFT - 1) / kFT;
  const float inv = 1.f / (4.f * (float)c->g.ncell * (float)nbatch);
  c->launches++;
  filter_grad_kernel<<<dim3(ntx * ntz, nbatch), kThreads, sizeof(TrainSmem), c->stream>>>(
      c->g, fp, wt, m, tg, inv, grad, loss);
  return cudaGetLastError();
}

__global__ void interleave4_kernel(int64_t ncell, int nb, const float *in, float4 *out) {
  const int64_t total = ncell * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = t / ncell, c = t - b * ncell;
    const float *src = in + b * 4 * ncell;
    out[t] = make_float4(src[c], src[ncell + c], src[2 * ncell + c], src[3 * ncell + c]);
  }
}

cudaError_t launch_interleave4(hv_ctx *c, int nb, const float *in, float4 *out) {
  const int64_t total = (int64_t)c->g.ncell * nb;
  const int blocks = (int)((total + 255) / 256 < 8192 ? (total + 255) / 256 : 8192);
  c->launches++;
  interleave4_kernel<<<blocks, 256, 0, c->stream>>>(c->g.ncell, nb, in, out);
  return cudaGetLastError();
}

cudaError_t launch_adam(hv_ctx *c, float *P, float *grad, float *m1, float *m2, int t, float lr,
                        const FilterParams &fp, __nv_bfloat16 *wt) {
  c->launches++;
  adam_kernel<<<14, 256, 0, c->stream>>>(P, grad, m1, m2, t, lr, fp.w, fp.bias, wt);
  return cudaGetLastError();
}

}  // namespace hv
