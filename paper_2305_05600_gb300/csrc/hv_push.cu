// Particle kernel of the hybrid PIC step: field gather at x^n, Boris push
// (Sec. 2.2, Eq. 9), deposit of n and J_i at the half-step position
// (App. B, Eqs. 13 and 17), move to x^{n+1} (Eq. 10) and the FP32-Kahan /
// FP64 block partials of the kinetic energy and momentum.
//
// Layout: SoA float32 particles, one thread owns 4 consecutive particles
// and moves them with 128-bit streaming loads/stores.  Fields are gathered
// from a ghost-padded array holding {Ex,Ey,Ez,Bx},{By,Bz,-,-} per cell (32 B,
// one sector).  Deposits are aggregated before they reach global memory:
// first in registers over a thread's 4 particles, then across the warp by a
// shuffle reduce-scatter over the lanes that share a deposit key (ions are
// sorted by cell, so a warp's 128 particles usually span one or two cells),
// and only then added to the padded accumulator with global reductions.
#include "hv_internal.cuh"

namespace hv {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct PushArgs {
  Soa s;
  int64_t n;
  const float4 *EB;
  float4 *acc;
  Geom g;
  PushConsts k;
  double *part;  // [gridDim.x][4]
  int *err;
};

template <int DIM, int SHAPE>
struct Shape {
  static constexpr int NT = SHAPE == 0 ? 1 : (SHAPE == 1 ? (DIM == 2 ? 5 : 7) : (DIM == 2 ? 4 : 8));
};

// Padded-index offset of target t from the key cell.
template <int DIM, int SHAPE>
__device__ __forceinline__ int target_off(int t, const Geom &g) {
  if (SHAPE == 0) return 0;
  if (SHAPE == 1) {
    if (DIM == 2) {
      return t == 0 ? 0 : t == 1 ? 1 : t == 2 ? -1 : t == 3 ? g.sz : -g.sz;
    }
    return t == 0 ? 0 : t == 1 ? 1 : t == 2 ? -1 : t == 3 ? g.sy : t == 4 ? -g.sy
           : t == 5 ? g.sz : -g.sz;
  }
  // CIC: base + {0,1} x {0,sy} x {0,sz}
  if (DIM == 2) return (t & 1) + ((t >> 1) & 1) * g.sz;
  return (t & 1) + ((t >> 1) & 1) * g.sy + ((t >> 2) & 1) * g.sz;
}

// Shape weights at relative coordinates (dx,dy,dz); returns the padded-index
// shift from the particle's cell to the key cell (non-zero only for CIC,
// whose 2^D stencil starts at the lower neighbour when d < 0).
template <int DIM, int SHAPE>
__device__ __forceinline__ int shape_weights(float dx, float dy, float dz, const Geom &g,
                                             float *wt) {
  if (SHAPE == 0) {
    wt[0] = 1.f;  // NGP (Eq. 13)
    return 0;
  }
  if (SHAPE == 1) {
    // QS (Eq. 17).  In the x-z layout the two y neighbours of a single-cell y
    // axis fold onto the cell: (3 - d^2)/6 + 2/12 = (4 - dx^2 - dz^2)/6.
    const float c6 = 1.f / 6.f, c12 = 1.f / 12.f;
    const float ax = 1.f + dx, bx = 1.f - dx, az = 1.f + dz, bz = 1.f - dz;
    if (DIM == 2) {
      wt[0] = (4.f - dx * dx - dz * dz) * c6;
      wt[1] = ax * ax * c12;
      wt[2] = bx * bx * c12;
      wt[3] = az * az * c12;
      wt[4] = bz * bz * c12;
    } else {
      const float ay = 1.f + dy, by = 1.f - dy;
      wt[0] = (3.f - dx * dx - dy * dy - dz * dz) * c6;
      wt[1] = ax * ax * c12;
      wt[2] = bx * bx * c12;
      wt[3] = ay * ay * c12;
      wt[4] = by * by * c12;
      wt[5] = az * az * c12;
      wt[6] = bz * bz * c12;
    }
    return 0;
  }
  // CIC on cell centres: per axis 1 - |d|/2 to the own cell, |d|/2 to the
  // neighbour on the side of d, written from the stencil base cell.
  const float fx = dx >= 0.f ? 0.5f * dx : 1.f + 0.5f * dx;
  const float fz = dz >= 0.f ? 0.5f * dz : 1.f + 0.5f * dz;
  int shift = (dx < 0.f ? -1 : 0) + (dz < 0.f ? -g.sz : 0);
  if (DIM == 2) {
    wt[0] = (1.f - fx) * (1.f - fz);
    wt[1] = fx * (1.f - fz);
    wt[2] = (1.f - fx) * fz;
    wt[3] = fx * fz;
  } else {
    const float fy = dy >= 0.f ? 0.5f * dy : 1.f + 0.5f * dy;
    shift += dy < 0.f ? -g.sy : 0;
    const float gx[2] = {1.f - fx, fx}, gy[2] = {1.f - fy, fy}, gz[2] = {1.f - fz, fz};
#pragma unroll
    for (int t = 0; t < 8; ++t) wt[t] = gx[t & 1] * gy[(t >> 1) & 1] * gz[(t >> 2) & 1];
  }
  return shift;
}

__device__ __forceinline__ void red_v4(float4 *addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}

__device__ __forceinline__ void red_f32(float *addr, float a) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(a) : "memory");
}

// Wrap a cell index that moved by at most one cell.
__device__ __forceinline__ int wrap1(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Shift a relative coordinate back into [-1, 1) after a move of less than
// one cell width on either side; the subtraction of 2 is exact (Sterbenz).
__device__ __forceinline__ int rebase(float &d) {
  const int m = (d >= 1.f) - (d < -1.f);
  d -= 2.f * (float)m;
  return m;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// Reduce-scatter of 32 values across the warp: afterwards lane l holds the
// warp sum of v[l].
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < o; ++j) {
      const float send = up ? v[j] : v[j + o];
      const float keep = up ? v[j + o] : v[j];
      v[j] = keep + __shfl_xor_sync(kFull, send, o);
    }
  }
  return v[0];
}

// MODE 0: full step.  MODE 1: start-up deposit at the current position with
// the stored velocity (no push, no move, no write-back).
template <int DIM, int SHAPE, int MODE>
__global__ void __launch_bounds__(256) push_kernel(PushArgs a) {
  constexpr int NT = Shape<DIM, SHAPE>::NT;
  constexpr int NV = NT * 4;
  static_assert(NV <= 32, "deposit vector must fit one warp");
  const Geom &g = a.g;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;

  float ks[4] = {0.f, 0.f, 0.f, 0.f}, kc[4] = {0.f, 0.f, 0.f, 0.f};

  const int64_t nq = (a.n + 3) >> 2;
  // contiguous range of quads per block (multiple of 32: whole warps)
  int64_t per = (nq + gridDim.x - 1) / gridDim.x;
  per = (per + 31) & ~int64_t(31);
  const int64_t qb = (int64_t)blockIdx.x * per;
  const int64_t qe = min(nq, qb + per);
  const bool mx = g.nx > 1, my = DIM == 3 && g.ny > 1, mz = g.nz > 1;

  for (int64_t q0 = qb + (int64_t)warp * 32; q0 < qe; q0 += (int64_t)nwarps * 32) {
    const int64_t q = q0 + lane;
    const bool has = q < qe;
    int4 c4 = make_int4(0, 0, 0, 0);
    float4 X = make_float4(0.f, 0.f, 0.f, 0.f), Y = X, Z = X, VX = X, VY = X, VZ = X, W = X;
    if (has) {
      c4 = __ldcs(reinterpret_cast<const int4 *>(a.s.cell) + q);
      X = __ldcs(reinterpret_cast<const float4 *>(a.s.ox) + q);
      if (DIM == 3) Y = __ldcs(reinterpret_cast<const float4 *>(a.s.oy) + q);
      Z = __ldcs(reinterpret_cast<const float4 *>(a.s.oz) + q);
      VX = __ldcs(reinterpret_cast<const float4 *>(a.s.vx) + q);
      VY = __ldcs(reinterpret_cast<const float4 *>(a.s.vy) + q);
      VZ = __ldcs(reinterpret_cast<const float4 *>(a.s.vz) + q);
      W = __ldcs(reinterpret_cast<const float4 *>(a.s.w) + q);
    }
    int cc[4] = {c4.x, c4.y, c4.z, c4.w};
    float ox[4] = {X.x, X.y, X.z, X.w}, oy[4] = {Y.x, Y.y, Y.z, Y.w},
          oz[4] = {Z.x, Z.y, Z.z, Z.w};
    float vx[4] = {VX.x, VX.y, VX.z, VX.w}, vy[4] = {VY.x, VY.y, VY.z, VY.w},
          vz[4] = {VZ.x, VZ.y, VZ.z, VZ.w};
    const float ww[4] = {W.x, W.y, W.z, W.w};

    float accv[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) accv[j] = 0.f;
    int key = -1;

#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const bool valid = has && (q * 4 + p) < a.n;
      if (!valid) continue;
      // decode the cell (indices are validated at load; a corrupt one is
      // latched and skipped rather than dereferenced)
      const uint32_t c = (uint32_t)cc[p];
      if (c >= (uint32_t)g.ncell) {
        atomicOr(a.err, kErrIndex);
        continue;
      }
      int i, j = 0, k;
      if (DIM == 2) {
        k = (int)fdiv(c, g.div_nx);
        i = (int)c - k * g.nx;
      } else {
        const int qq = (int)fdiv(c, g.div_nx);
        i = (int)c - qq * g.nx;
        k = (int)fdiv((uint32_t)qq, g.div_ny);
        j = qq - k * g.ny;
      }
      const float dy0 = DIM == 3 ? oy[p] : 0.f;
      float vxp = vx[p], vyp = vy[p], vzp = vz[p];

      if (MODE == 0) {
        // gather E^n, B^n at x^n (same weights as the deposit)
        float wt[NT];
        const int kshift = shape_weights<DIM, SHAPE>(ox[p], dy0, oz[p], g, wt);
        const int pc = (i + 1) + (DIM == 3 ? (j + 1) * g.sy : 0) + (k + 1) * g.sz + kshift;
        float ex = 0.f, ey = 0.f, ez = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const int pt = pc + target_off<DIM, SHAPE>(t, g);
          const float4 f0 = __ldg(a.EB + 2 * pt);
          const float4 f1 = __ldg(a.EB + 2 * pt + 1);
          ex = fmaf(wt[t], f0.x, ex);
          ey = fmaf(wt[t], f0.y, ey);
          ez = fmaf(wt[t], f0.z, ez);
          bx = fmaf(wt[t], f0.w, bx);
          by = fmaf(wt[t], f1.x, by);
          bz = fmaf(wt[t], f1.y, bz);
        }
        // Boris: half E kick, rotation, half E kick (Eq. 9)
        const float h = a.k.qmdt2;
        const float vmx = vxp + h * ex, vmy = vyp + h * ey, vmz = vzp + h * ez;
        const float tx = h * bx, ty = h * by, tz = h * bz;
        const float f = 2.f / (1.f + (tx * tx + ty * ty + tz * tz));
        const float sx = f * tx, sy = f * ty, sz = f * tz;
        const float vpx = vmx + (vmy * tz - vmz * ty);
        const float vpy = vmy + (vmz * tx - vmx * tz);
        const float vpz = vmz + (vmx * ty - vmy * tx);
        vxp = vmx + (vpy * sz - vpz * sy) + h * ex;
        vyp = vmy + (vpz * sx - vpx * sz) + h * ey;
        vzp = vmz + (vpx * sy - vpy * sx) + h * ez;
      }

      // half-step and full-step positions (Eq. 10, App. B)
      float hx = ox[p], hy = dy0, hz = oz[p];
      float nxo = ox[p], nyo = dy0, nzo = oz[p];
      int ih = i, jh = j, kh = k, in_ = i, jn = j, kn = k;
      if (MODE == 0) {
        bool ok = true;
        if (mx) {
          hx = ox[p] + vxp * a.k.cx;
          nxo = ox[p] + vxp * (2.f * a.k.cx);
          ok = ok && fabsf(nxo) < 3.f;
        }
        if (my) {
          hy = dy0 + vyp * a.k.cy;
          nyo = dy0 + vyp * (2.f * a.k.cy);
          ok = ok && fabsf(nyo) < 3.f;
        }
        if (mz) {
          hz = oz[p] + vzp * a.k.cz;
          nzo = oz[p] + vzp * (2.f * a.k.cz);
          ok = ok && fabsf(nzo) < 3.f;
        }
        if (!ok) {
          // more than one cell per step or non-finite: latch and freeze
          atomicOr(a.err, isfinite(vxp + vyp + vzp) ? kErrCfl : kErrNonFinite);
          hx = nxo = ox[p];
          hy = nyo = dy0;
          hz = nzo = oz[p];
          vxp = vx[p];
          vyp = vy[p];
          vzp = vz[p];
        } else {
          ih = wrap1(i + rebase(hx), g.nx);
          in_ = wrap1(i + rebase(nxo), g.nx);
          if (DIM == 3) {
            jh = wrap1(j + rebase(hy), g.ny);
            jn = wrap1(j + rebase(nyo), g.ny);
          }
          kh = wrap1(k + rebase(hz), g.nz);
          kn = wrap1(k + rebase(nzo), g.nz);
        }
        // write back into the quad registers
        cc[p] = in_ + g.nx * (jn + g.ny * kn);
        ox[p] = nxo;
        if (DIM == 3) oy[p] = nyo;
        oz[p] = nzo;
        vx[p] = vxp;
        vy[p] = vyp;
        vz[p] = vzp;
      }

      // deposit q w S / V_c and q w v S / V_c at the half-step position
      float wt[NT];
      const int kshift = shape_weights<DIM, SHAPE>(hx, hy, hz, g, wt);
      const int pk = (ih + 1) + (DIM == 3 ? (jh + 1) * g.sy : 0) + (kh + 1) * g.sz + kshift;
      const float s = a.k.qvc * ww[p];
      float cv[NV];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const float st = wt[t] * s;
        cv[4 * t + 0] = st;
        cv[4 * t + 1] = st * vxp;
        cv[4 * t + 2] = st * vyp;
        cv[4 * t + 3] = st * vzp;
      }
      if (key < 0 || pk == key) {
        key = pk;
#pragma unroll
        for (int jv = 0; jv < NV; ++jv) accv[jv] += cv[jv];
      } else {
#pragma unroll
        for (int t = 0; t < NT; ++t)
          red_v4(a.acc + pk + target_off<DIM, SHAPE>(t, g), cv[4 * t], cv[4 * t + 1],
                 cv[4 * t + 2], cv[4 * t + 3]);
      }
      if (MODE == 0) {
        const float mw = a.k.mass * ww[p];
        kahan_add(ks[0], kc[0], 0.5f * mw * (vxp * vxp + vyp * vyp + vzp * vzp));
        kahan_add(ks[1], kc[1], mw * vxp);
        kahan_add(ks[2], kc[2], mw * vyp);
        kahan_add(ks[3], kc[3], mw * vzp);
      }
    }

    if (MODE == 0 && has) {
      __stcs(reinterpret_cast<int4 *>(a.s.cell) + q, make_int4(cc[0], cc[1], cc[2], cc[3]));
      __stcs(reinterpret_cast<float4 *>(a.s.ox) + q, make_float4(ox[0], ox[1], ox[2], ox[3]));
      if (DIM == 3)
        __stcs(reinterpret_cast<float4 *>(a.s.oy) + q, make_float4(oy[0], oy[1], oy[2], oy[3]));
      __stcs(reinterpret_cast<float4 *>(a.s.oz) + q, make_float4(oz[0], oz[1], oz[2], oz[3]));
      __stcs(reinterpret_cast<float4 *>(a.s.vx) + q, make_float4(vx[0], vx[1], vx[2], vx[3]));
      __stcs(reinterpret_cast<float4 *>(a.s.vy) + q, make_float4(vy[0], vy[1], vy[2], vy[3]));
      __stcs(reinterpret_cast<float4 *>(a.s.vz) + q, make_float4(vz[0], vz[1], vz[2], vz[3]));
    }

    // warp aggregation: lanes sharing a key are summed by a reduce-scatter;
    // lane l then owns value l = (target l/4, channel l%4) of that key.
    unsigned pending = __ballot_sync(kFull, key >= 0);
    int rounds = 0;
    while (pending) {
      if (rounds == 3) {
        // many distinct keys in this warp: the rest add their own sums
        if (key >= 0 && ((pending >> lane) & 1u)) {
#pragma unroll
          for (int t = 0; t < NT; ++t)
            red_v4(a.acc + key + target_off<DIM, SHAPE>(t, g), accv[4 * t], accv[4 * t + 1],
                   accv[4 * t + 2], accv[4 * t + 3]);
        }
        break;
      }
      const int leader = __ffs(pending) - 1;
      const int lkey = __shfl_sync(kFull, key, leader);
      const unsigned peers = __ballot_sync(kFull, key == lkey);
      const bool mine = (peers >> lane) & 1u;
      float v[32];
#pragma unroll
      for (int jv = 0; jv < 32; ++jv) v[jv] = (jv < NV && mine) ? accv[jv] : 0.f;
      const float tot = reduce_scatter32(v, lane);
      if (lane < NV) {
        const int t = lane >> 2;
        float *dst = reinterpret_cast<float *>(a.acc + lkey + target_off<DIM, SHAPE>(t, g)) +
                     (lane & 3);
        red_f32(dst, tot);
      }
      pending &= ~peers;
      ++rounds;
    }
  }

  if (MODE == 0) {
    // FP64 block partials of W_K and P (deterministic order)
    __shared__ double red[8][4];
    double d[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      d[m] = (double)ks[m] - (double)kc[m];
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) d[m] += __shfl_xor_sync(kFull, d[m], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int m = 0; m < 4; ++m) red[warp][m] = d[m];
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      double s = 0.0;
      for (int w = 0; w < nwarps; ++w) s += red[w][threadIdx.x];
      a.part[(int64_t)blockIdx.x * 4 + threadIdx.x] = s;
    }
  }
}

template <int DIM, int SHAPE, int MODE>
cudaError_t launch_t(const PushArgs &a, int blocks, cudaStream_t s) {
  push_kernel<DIM, SHAPE, MODE><<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <int DIM, int MODE>
cudaError_t launch_shape(int shape, const PushArgs &a, int blocks, cudaStream_t s) {
  switch (shape) {
    case 0: return launch_t<DIM, 0, MODE>(a, blocks, s);
    case 1: return launch_t<DIM, 1, MODE>(a, blocks, s);
    default: return launch_t<DIM, 2, MODE>(a, blocks, s);
  }
}

}  // namespace

int push_grid_blocks(int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, push_kernel<2, 1, 0>, 256, 0);
  if (per < 1) per = 1;
  if (sms < 1) sms = 1;
  return sms * per;
}

cudaError_t launch_push(hv_ctx *c, int species, int mode) {
  Species &sp = c->sp[species];
  if (sp.n == 0) return cudaSuccess;
  PushArgs a;
  a.s = sp.buf[sp.cur];
  a.n = sp.n;
  a.EB = c->EB;
  a.acc = c->acc;
  a.g = c->g;
  a.k.qmdt2 = (float)(0.5 * sp.q / sp.m * c->p.dt);
  a.k.cx = c->g.nx > 1 ? (float)(c->p.dt / c->p.dx) : 0.f;
  a.k.cy = c->g.ny > 1 ? (float)(c->p.dt / c->p.dy) : 0.f;
  a.k.cz = c->g.nz > 1 ? (float)(c->p.dt / c->p.dz) : 0.f;
  a.k.qvc = (float)(sp.q / c->vc);
  a.k.mass = (float)sp.m;
  a.part = c->pushpart + (size_t)species * c->push_blocks * 4;
  a.err = c->err;
  c->launches++;
  const int shape = c->p.shape;
  if (c->g.dim2) {
    return mode == 0 ? launch_shape<2, 0>(shape, a, c->push_blocks, c->stream)
                     : launch_shape<2, 1>(shape, a, c->push_blocks, c->stream);
  }
  return mode == 0 ? launch_shape<3, 0>(shape, a, c->push_blocks, c->stream)
                   : launch_shape<3, 1>(shape, a, c->push_blocks, c->stream);
}

}  // namespace hv
