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

}  // namespace

size_t filter_smem_bytes() { return sizeof(Smem); }

cudaError_t launch_filter(hv_ctx *c, const FilterParams &fp, const float4 *in, float4 *out) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(filter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(Smem));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
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

}  // namespace hv
