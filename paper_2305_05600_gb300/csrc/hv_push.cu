// Particle kernel of the hybrid PIC step: field gather at x^n, Boris push
// (Sec. 2.2, Eq. 9), deposit of n and J_i at the half-step position
// (App. B, Eqs. 13 and 17), move to x^{n+1} (Eq. 10), and FP32-Kahan /
// FP64 block partials of the kinetic energy and momentum.
//
// Layout: SoA float32 ions whose cell is stored as a voxel index of the
// ghost-padded grid (two ghost layers), so no index decode or wrap is needed
// on the hot path: the half-step cell is the voxel plus the cell shift, the
// deposit stencil may reach into the ghost layers (folded back afterwards),
// and the new cell after the move is wrapped into the interior.  Ions move
// between global memory and per-warp shared staging buffers with bulk
// copies.  Fields are gathered from {Ex,Ey,Ez,Bx},{By,Bz,-,-} per voxel.
//
// Deposits are aggregated in registers before they reach global memory: a
// lane takes kChunk consecutive ions and sums their deposits per run of
// equal deposit key, flushing a run with vector reductions.  In the x-z
// layout each warp first counting-sorts its staging tile by cell in shared
// memory, so the runs stay long however far the ions have drifted since the
// last global sort.  For QS in the x-z layout the accumulated quantities are
// the per-cell moment sums s*(1, dx, dx^2, dz, dz^2) of Eq. 17's weights, so
// every ion of a cell contributes to one 80-byte record; the fold kernel
// applies the stencil.  For CIC, NGP and 3D QS the per-target contributions
// are accumulated.
#include <climits>

#include "hv_internal.cuh"

// Threads per block, resident blocks per SM the push kernel is compiled for
// (register budget 65536 / (threads * blocks)), and ions per lane per tile.
#ifndef HV_PUSH_THREADS
#define HV_PUSH_THREADS 256
#endif
#ifndef HV_PUSH_MIN_BLOCKS
#define HV_PUSH_MIN_BLOCKS 2
#endif
#ifndef HV_PUSH_CHUNK
#define HV_PUSH_CHUNK 8
#endif

namespace hv {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = HV_PUSH_THREADS;
constexpr int kChunk = HV_PUSH_CHUNK;  // consecutive ions per lane per tile
constexpr int kTile = 32 * kChunk;     // ions per warp tile

struct PushArgs {
  Soa s;
  int64_t n;
  const int *tile_off;  // [ntiles + 1]
  const float4 *EB;
  float4 *acc;       // per-target accumulator
  float *accm;       // per-cell moment records (QS in the x-z layout)
  const int *wrapvox;
  Geom g;
  PushConsts k;
  double *part;      // [gridDim.x][4]
  int *err;
};

template <int DIM, int SHAPE>
struct Shape {
  static constexpr int NT = SHAPE == 0 ? 1 : (SHAPE == 1 ? (DIM == 2 ? 5 : 7) : (DIM == 2 ? 4 : 8));
  static constexpr bool REC = SHAPE == 1 && DIM == 2;  // moment records
  static constexpr int NV = REC ? kMono : NT * 4;
};

// Voxel offset of gather/deposit target t from the key voxel.
template <int DIM, int SHAPE>
__device__ __forceinline__ int target_off(int t, const Geom &g) {
  if (SHAPE == 0) return 0;
  if (SHAPE == 1) {
    if (DIM == 2) return t == 0 ? 0 : t == 1 ? 1 : t == 2 ? -1 : t == 3 ? g.sz : -g.sz;
    return t == 0 ? 0 : t == 1 ? 1 : t == 2 ? -1 : t == 3 ? g.sy : t == 4 ? -g.sy
           : t == 5 ? g.sz : -g.sz;
  }
  if (DIM == 2) return (t & 1) + ((t >> 1) & 1) * g.sz;
  return (t & 1) + ((t >> 1) & 1) * g.sy + ((t >> 2) & 1) * g.sz;
}

// Shape weights at relative coordinates (dx,dy,dz); returns the voxel shift
// from the particle's cell to the key voxel (non-zero only for CIC, whose
// 2^D stencil starts at the lower neighbour when d < 0).
template <int DIM, int SHAPE>
__device__ __forceinline__ int shape_weights(float dx, float dy, float dz, const Geom &g,
                                             float *wt) {
  if (SHAPE == 0) {
    wt[0] = 1.f;  // NGP (Eq. 13)
    return 0;
  }
  if (SHAPE == 1) {
    // QS (Eq. 17).  In the x-z layout the two y neighbours of the single y
    // cell fold onto the cell: (3 - |d|^2)/6 + 2/12 = (4 - dx^2 - dz^2)/6.
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

__device__ __forceinline__ void red_v4(float *addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}


// Shift a relative coordinate back into [-1, 1) after a move of less than
// one cell on either side; the subtraction of 2 is exact (Sterbenz).
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

// Deposit values of one ion: QS x-z records (moment sums) or per-target
// contributions, both NV floats.
template <int DIM, int SHAPE>
__device__ __forceinline__ int deposit_values(float hx, float hy, float hz, float s, float vx,
                                              float vy, float vz, const Geom &g, float *cv) {
  using S = Shape<DIM, SHAPE>;
  if (S::REC) {
    const float sx = s * hx, sz = s * hz;
    const float v3[3] = {vx, vy, vz};
    cv[0] = s;
    cv[1] = sx;
    cv[2] = sx * hx;
    cv[3] = sz;
    cv[4] = sz * hz;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float ta = s * v3[a];
      const float tx = ta * hx, tz = ta * hz;
      cv[5 * a + 5] = ta;
      cv[5 * a + 6] = tx;
      cv[5 * a + 7] = tx * hx;
      cv[5 * a + 8] = tz;
      cv[5 * a + 9] = tz * hz;
    }
    return 0;
  }
  float wt[S::NT];
  const int shift = shape_weights<DIM, SHAPE>(hx, hy, hz, g, wt);
#pragma unroll
  for (int t = 0; t < S::NT; ++t) {
    const float st = wt[t] * s;
    cv[4 * t + 0] = st;
    cv[4 * t + 1] = st * vx;
    cv[4 * t + 2] = st * vy;
    cv[4 * t + 3] = st * vz;
  }
  return shift;
}

// Add a lane's NV deposit values at `key` with vector reductions.
template <int DIM, int SHAPE>
__device__ __forceinline__ void flush_direct(const PushArgs &a, int key, const float *v) {
  using S = Shape<DIM, SHAPE>;
  if (S::REC) {
    float *rec = a.accm + (size_t)key * kMono;
#pragma unroll
    for (int q = 0; q < kMono / 4; ++q) red_v4(rec + 4 * q, v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
#pragma unroll
    for (int t = 0; t < S::NT; ++t)
      red_v4(reinterpret_cast<float *>(a.acc + key + target_off<DIM, SHAPE>(t, a.g)), v[4 * t],
             v[4 * t + 1], v[4 * t + 2], v[4 * t + 3]);
  }
}

// ----------------------------------------------------------------------------
// TMA bulk copies and mbarriers (inline PTX, sm_90+)
// ----------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bounded wait on a transaction barrier: gives up after a fixed number of
// polls (a copy that never lands would otherwise hang the GPU) and returns
// false so the caller can latch an error and stop.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 24); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Supercell window: the tile and a halo of RE cells.  Ions that drifted up
// to H cells out of their tile since the last sort still gather from the
// window in shared memory.
template <int DIM>
struct Win {
  static constexpr int TX = DIM == 2 ? kTile2X : kTile3;
  static constexpr int TY = DIM == 2 ? 1 : kTile3;
  static constexpr int TZ = DIM == 2 ? kTile2Z : kTile3;
  static constexpr int H = DIM == 2 ? 2 : 1;
  static constexpr int RE = H + 1;
  static constexpr int EX = TX + 2 * RE, EY = DIM == 2 ? 1 : TY + 2 * RE, EZ = TZ + 2 * RE;
  static constexpr int NEB = EX * EY * EZ;
};

// In the x-z layout every staging tile is counting-sorted by cell (the
// window cells, plus one bin for every other cell) before it is processed,
// so that a lane's consecutive ions share a deposit cell however far the
// ions have drifted from the order of the last global sort.
constexpr int kBins = 512;
static_assert(Win<2>::NEB < kBins, "window cells + overflow bin must fit the bins");
static_assert((kChunk & (kChunk - 1)) == 0 && kChunk <= 32, "chunk must be a power of two");

constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Shared-memory layout of one push block (one supercell tile).
//   stage: one kTile-ion staging buffer per warp (bulk-copied in and out)
//   hist, perm: per-warp bins and processing order (sorted layout only)
//   eb:    E, B of the window, 2 float4 per cell
template <int DIM, int SHAPE>
struct Layout {
  static constexpr bool SORT = DIM == 2;
  static constexpr int NW = kThreads / 32;
  static constexpr int NA = DIM == 2 ? 7 : 8;  // cell, ox, [oy], oz, vx, vy, vz, w
  static constexpr size_t stage_bytes = (size_t)NA * kTile * 4;
  static constexpr size_t hist_bytes = SORT ? kBins * 4 : 0;
  static constexpr size_t perm_bytes = SORT ? align_up(kTile * 2, 16) : 0;
  static constexpr size_t off_hist = stage_bytes * NW;
  static constexpr size_t off_perm = off_hist + hist_bytes * NW;
  static constexpr size_t off_eb = align_up(off_perm + perm_bytes * NW, 16);
  static constexpr size_t off_bar = off_eb + (size_t)Win<DIM>::NEB * 32;
  static constexpr size_t bytes = off_bar + 8 * NW;
};

// Array slot of each particle field in a staging buffer.
template <int DIM>
struct Slot {
  static constexpr int CELL = 0, OX = 1, OY = DIM == 3 ? 2 : 1, OZ = DIM == 3 ? 3 : 2,
                       VX = OZ + 1, VY = OZ + 2, VZ = OZ + 3, W = OZ + 4;
};

template <int DIM>
__device__ __forceinline__ void soa_ptrs(const Soa &s, void **p) {
  p[Slot<DIM>::CELL] = s.cell;
  p[Slot<DIM>::OX] = s.ox;
  if (DIM == 3) p[Slot<DIM>::OY] = s.oy;
  p[Slot<DIM>::OZ] = s.oz;
  p[Slot<DIM>::VX] = s.vx;
  p[Slot<DIM>::VY] = s.vy;
  p[Slot<DIM>::VZ] = s.vz;
  p[Slot<DIM>::W] = s.w;
}

// Padded coordinates of a voxel.
__device__ __forceinline__ void voxel_coords(const Geom &g, int vox, int &ip, int &jp, int &kp) {
  const uint32_t q = fdiv((uint32_t)vox, g.div_px);
  ip = vox - (int)q * g.px;
  if (g.dim2) {
    jp = kGhost;
    kp = (int)q;
  } else {
    kp = (int)fdiv(q, g.div_py);
    jp = (int)q - kp * g.py;
  }
}

// Sort bin of a voxel in the x-z layout: its window cell, or the last bin.
__device__ __forceinline__ int sort_bin(const Geom &g, int vox, int i0, int k0) {
  using W = Win<2>;
  if (vox < g.vlo || vox >= g.vhi) return kBins - 1;
  int ip, jp, kp;
  voxel_coords(g, vox, ip, jp, kp);
  const int rx = ip - kGhost - i0 + W::RE, rz = kp - kGhost - k0 + W::RE;
  return ((unsigned)rx < (unsigned)W::EX && (unsigned)rz < (unsigned)W::EZ) ? rx + rz * W::EX
                                                                          : kBins - 1;
}

// One ion of the step: gather E^n, B^n at x^n, Boris push, move to x^{n+1}
// (MODE 0; the state is updated in place and the kinetic-energy/momentum
// terms are added to rk), then the deposit values at the half-step
// position.  Returns the voxel of the deposit key, or INT_MIN for a corrupt
// cell index (latched in the error word; the ion is left as it is).
template <int DIM, int SHAPE, int MODE>
__device__ __forceinline__ int push_ion(const PushArgs &a, const float4 *eb, int i0, int j0,
                                        int k0, int &vox, float &ox, float &oy, float &oz,
                                        float &vx, float &vy, float &vz, float w, float *cv,
                                        float *rk) {
  using W = Win<DIM>;
  constexpr int NT = Shape<DIM, SHAPE>::NT;
  const Geom &g = a.g;
  const int vox0 = vox;
  if (vox0 < g.vlo || vox0 >= g.vhi) {
    atomicOr(a.err, kErrIndex);
    return INT_MIN;
  }
  // cell relative to the tile; in the window if within H of the tile
  int ip, jp, kp;
  voxel_coords(g, vox0, ip, jp, kp);
  const int rx = ip - kGhost - i0, rz = kp - kGhost - k0;
  const int ry = DIM == 2 ? 0 : jp - kGhost - j0;
  const bool inwin = rx >= -W::H && rx < W::TX + W::H && rz >= -W::H && rz < W::TZ + W::H &&
                     (DIM == 2 || (ry >= -W::H && ry < W::TY + W::H));
  const int eslot = (rx + W::RE) + (DIM == 2 ? 0 : (ry + W::RE) * W::EX) +
                    (rz + W::RE) * W::EX * W::EY;
  const float dy0 = DIM == 3 ? oy : 0.f;
  float vxp = vx, vyp = vy, vzp = vz;
  float hx = ox, hy = dy0, hz = oz;
  int shx = 0, shy = 0, shz = 0;

  if (MODE == 0) {
    // gather E^n, B^n at x^n with the deposit's weights (App. B)
    float wt[NT];
    const int ks_ = shape_weights<DIM, SHAPE>(ox, dy0, oz, g, wt);
    float ex = 0.f, ey = 0.f, ez = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
    if (inwin) {
      // window offset of the stencil base (CIC may start one cell lower)
      int eb0 = eslot;
      if (SHAPE == 2) {
        eb0 += (ox < 0.f ? -1 : 0) + (oz < 0.f ? -W::EX * W::EY : 0);
        if (DIM == 3) eb0 += dy0 < 0.f ? -W::EX : 0;
      }
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        int wo;
        if (SHAPE == 0) wo = 0;
        else if (SHAPE == 1)
          wo = DIM == 2 ? (t == 0 ? 0 : t == 1 ? 1 : t == 2 ? -1 : t == 3 ? W::EX : -W::EX)
                        : (t == 0 ? 0 : t == 1 ? 1 : t == 2 ? -1 : t == 3 ? W::EX
                           : t == 4 ? -W::EX : t == 5 ? W::EX * W::EY : -W::EX * W::EY);
        else
          wo = DIM == 2 ? (t & 1) + ((t >> 1) & 1) * W::EX
                        : (t & 1) + ((t >> 1) & 1) * W::EX + ((t >> 2) & 1) * W::EX * W::EY;
        const float4 f0 = eb[2 * (eb0 + wo)];
        const float4 f1 = eb[2 * (eb0 + wo) + 1];
        ex = fmaf(wt[t], f0.x, ex);
        ey = fmaf(wt[t], f0.y, ey);
        ez = fmaf(wt[t], f0.z, ez);
        bx = fmaf(wt[t], f0.w, bx);
        by = fmaf(wt[t], f1.x, by);
        bz = fmaf(wt[t], f1.y, bz);
      }
    } else {
      const int pc = vox0 + ks_;
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

    // half-step and full-step positions (Eq. 10; App. B); the
    // displacement coefficients are 0 along single-cell axes
    hx = ox + vxp * a.k.cx;
    hz = oz + vzp * a.k.cz;
    float nxo = ox + vxp * (2.f * a.k.cx);
    float nzo = oz + vzp * (2.f * a.k.cz);
    float nyo = dy0;
    bool ok = fabsf(nxo) < 3.f && fabsf(nzo) < 3.f;
    if (DIM == 3) {
      hy = dy0 + vyp * a.k.cy;
      nyo = dy0 + vyp * (2.f * a.k.cy);
      ok = ok && fabsf(nyo) < 3.f;
    }
    if (!ok) {
      // more than one cell in a step, or non-finite: latch and freeze
      atomicOr(a.err, isfinite(vxp + vyp + vzp) ? kErrCfl : kErrNonFinite);
      hx = nxo = ox;
      hy = nyo = dy0;
      hz = nzo = oz;
      vxp = vx;
      vyp = vy;
      vzp = vz;
    }
    shx = rebase(hx);
    shz = rebase(hz);
    const int mx = rebase(nxo), mz = rebase(nzo);
    int my = 0;
    if (DIM == 3) {
      shy = rebase(hy);
      my = rebase(nyo);
    }
    // new cell, wrapped into the interior
    const int i1 = ip - kGhost + mx, k1 = kp - kGhost + mz;
    const int j1 = DIM == 2 ? 0 : jp - kGhost + my;
    const int iw = i1 < 0 ? i1 + g.nx : (i1 >= g.nx ? i1 - g.nx : i1);
    const int kw = k1 < 0 ? k1 + g.nz : (k1 >= g.nz ? k1 - g.nz : k1);
    const int jw = DIM == 2 ? 0 : (j1 < 0 ? j1 + g.ny : (j1 >= g.ny ? j1 - g.ny : j1));
    vox = voxel_of(g, iw, jw, kw);
    ox = nxo;
    if (DIM == 3) oy = nyo;
    oz = nzo;
    vx = vxp;
    vy = vyp;
    vz = vzp;
    const float mw = a.k.mass * w;
    rk[0] += 0.5f * mw * (vxp * vxp + vyp * vyp + vzp * vzp);
    rk[1] += mw * vxp;
    rk[2] += mw * vyp;
    rk[3] += mw * vzp;
  }

  // deposit q w S / V_c and q w v S / V_c at the half-step position
  const int kshift = deposit_values<DIM, SHAPE>(hx, hy, hz, a.k.qvc * w, vxp, vyp, vzp, g, cv);
  return vox0 + shx + shz * g.sz + (DIM == 3 ? shy * g.sy : 0) + kshift;
}

// A lane's register run: the deposit values summed over consecutive ions
// with the same deposit key.  For QS and NGP (keys are cells) an ion that
// left the run's cell is flushed on its own while the run continues; a new
// run starts only with an ion whose key is its own cell.
template <int DIM, int SHAPE>
struct Run {
  static constexpr int NV = Shape<DIM, SHAPE>::NV;
  static constexpr bool CELLKEY = SHAPE != 2;
  int key;
  float acc[NV];

  __device__ __forceinline__ void reset() {
    key = INT_MIN;
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = 0.f;
  }
  __device__ __forceinline__ void add(const PushArgs &a, int pk, int own, const float *cv) {
    if (pk == key) {
#pragma unroll
      for (int j = 0; j < NV; ++j) acc[j] += cv[j];
    } else if (!CELLKEY || pk == own || key == INT_MIN) {
      if (key != INT_MIN) flush_direct<DIM, SHAPE>(a, key, acc);
      key = pk;
#pragma unroll
      for (int j = 0; j < NV; ++j) acc[j] = cv[j];
    } else {
      flush_direct<DIM, SHAPE>(a, pk, cv);
    }
  }
  __device__ __forceinline__ void finish(const PushArgs &a) {
    if (key != INT_MIN) flush_direct<DIM, SHAPE>(a, key, acc);
    key = INT_MIN;
  }
};

// MODE 0: full step.  MODE 1: start-up deposit at the current position with
// the stored velocity (no push, no move, no write-back).
//
// One block per supercell tile.  Ions are kept sorted tile-major, so the
// block's ion range [tile_off[t], tile_off[t+1]) (rounded to whole quads)
// lies in the tile, give or take the drift since the last sort.  The block
// stages E and B of the tile and a halo in shared memory; ions that drifted
// further gather from global memory.  Each warp streams tiles of kTile ions
// through shared memory with bulk copies.  In the x-z layout the warp
// counting-sorts each staging tile by cell and each lane takes kChunk
// consecutive ions of that order; in 3D each lane takes kChunk consecutive
// ions of the memory order.  A lane sums the deposits of its ions in
// registers per run of equal deposit key, flushing a run with vector
// reductions into the global accumulator.
template <int DIM, int SHAPE, int MODE>
__global__ void __launch_bounds__(kThreads, HV_PUSH_MIN_BLOCKS) push_kernel(PushArgs a) {
  using L = Layout<DIM, SHAPE>;
  using W = Win<DIM>;
  using SL = Slot<DIM>;
  constexpr int NV = Shape<DIM, SHAPE>::NV;
  constexpr int NA = L::NA;
  constexpr int CQ = kChunk / 4;  // quads per lane per staging tile
  constexpr int TQ = kTile / 4;   // quads per staging tile
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Geom &g = a.g;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int nwarps = kThreads / 32;
  float(&T)[NA][kTile] = *reinterpret_cast<float(*)[NA][kTile]>(smem_raw + L::stage_bytes * warp);
  int(&TC)[NA][kTile] = *reinterpret_cast<int(*)[NA][kTile]>(smem_raw + L::stage_bytes * warp);
  float4 *eb = reinterpret_cast<float4 *>(smem_raw + L::off_eb);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + L::off_bar) + warp;

  // tile origin and the block's range of quads
  const int tile = blockIdx.x;
  const int ti = tile % g.ntx, tj = (tile / g.ntx) % g.nty, tk = tile / (g.ntx * g.nty);
  const int i0 = ti * W::TX, j0 = tj * W::TY, k0 = tk * W::TZ;
  const int64_t nq = (a.n + 3) >> 2;
  const int64_t qa = tile == 0 ? 0 : (int64_t)a.tile_off[tile] >> 2;
  const int64_t qe = tile == g.ntiles - 1 ? nq : (int64_t)a.tile_off[tile + 1] >> 2;

  // stage E, B of the window
  if (MODE == 0) {
    for (int c = threadIdx.x; c < W::NEB; c += kThreads) {
      const int wx = c % W::EX, wy = (c / W::EX) % W::EY, wz = c / (W::EX * W::EY);
      const int ip = i0 + wx - W::RE + kGhost, kp = k0 + wz - W::RE + kGhost;
      const int jp = DIM == 2 ? 0 : j0 + wy - W::RE + kGhost;
      if (ip < 0 || ip >= g.px || kp < 0 || kp >= g.pz || (DIM == 3 && (jp < 0 || jp >= g.py)))
        continue;  // outside the padded grid: never read by an in-window ion
      const int v = ip + (DIM == 2 ? 0 : jp * g.sy) + kp * g.sz;
      eb[2 * c] = __ldg(a.EB + 2 * v);
      eb[2 * c + 1] = __ldg(a.EB + 2 * v + 1);
    }
  }
  if (lane == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  float ks[4] = {0.f, 0.f, 0.f, 0.f}, kc[4] = {0.f, 0.f, 0.f, 0.f};
  void *gp[8];
  soa_ptrs<DIM>(a.s, gp);
  bool failed = false;
  int k = 0;
  const int64_t nst = qe > qa ? (qe - qa + TQ - 1) / TQ : 0;  // staging tiles

  for (int64_t st = warp; st < nst && !failed; st += nwarps, ++k) {
    const int64_t q0 = qa + st * TQ;
    const int nqt = (int)min((int64_t)TQ, qe - q0);
    if (lane == 0) {
      bulk_wait_read_all();  // the previous store has read the buffer
      const uint32_t bytes = (uint32_t)nqt * 16u;
      mbar_expect_tx(bar, bytes * NA);
#pragma unroll
      for (int f = 0; f < NA; ++f)
        bulk_load(T[f], reinterpret_cast<const char *>(gp[f]) + q0 * 16, bytes, bar);
    }
    if (!mbar_wait_bounded(bar, (uint32_t)(k & 1))) {
      failed = true;
      mbar_wait_bounded(bar, (uint32_t)(k & 1));  // one more bounded chance
      break;
    }

    Run<DIM, SHAPE> run;
    run.reset();
    float rk[4] = {0.f, 0.f, 0.f, 0.f};

    if constexpr (L::SORT) {
      int *hist = reinterpret_cast<int *>(smem_raw + L::off_hist + L::hist_bytes * warp);
      uint16_t *perm = reinterpret_cast<uint16_t *>(smem_raw + L::off_perm + L::perm_bytes * warp);
      const int nion = (int)min((int64_t)nqt * 4, a.n - q0 * 4);
      // lanes start their chunk at a rotated ion so that a warp's shared
      // loads of one field hit distinct banks
      const int rot = lane / (32 / kChunk);
#pragma unroll
      for (int b = lane * 4; b < kBins; b += 128)
        *reinterpret_cast<int4 *>(hist + b) = make_int4(0, 0, 0, 0);
      __syncwarp();
      // bin of every ion and its rank in the bin
      uint32_t br[kChunk];
#pragma unroll
      for (int j = 0; j < kChunk; ++j) {
        const int e = lane * kChunk + ((j + rot) & (kChunk - 1));
        br[j] = 0xffffffffu;
        if (e < nion) {
          const int bin = sort_bin(g, TC[SL::CELL][e], i0, k0);
          const int r = atomicAdd(hist + bin, 1);
          br[j] = ((uint32_t)bin << 16) | (uint32_t)r;
        }
      }
      __syncwarp();
      // exclusive scan of the bins: each lane owns kBins / 32 consecutive bins
      {
        constexpr int PB = kBins / 32;
        int v[PB];
        int4 *h4 = reinterpret_cast<int4 *>(hist + lane * PB);
#pragma unroll
        for (int q = 0; q < PB / 4; ++q) {
          const int4 x = h4[q];
          v[4 * q] = x.x;
          v[4 * q + 1] = x.y;
          v[4 * q + 2] = x.z;
          v[4 * q + 3] = x.w;
        }
        int tot = 0;
#pragma unroll
        for (int q = 0; q < PB; ++q) {
          const int t = v[q];
          v[q] = tot;
          tot += t;
        }
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl += y;
        }
        const int base = incl - tot;
#pragma unroll
        for (int q = 0; q < PB / 4; ++q)
          h4[q] = make_int4(v[4 * q] + base, v[4 * q + 1] + base, v[4 * q + 2] + base,
                            v[4 * q + 3] + base);
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < kChunk; ++j) {
        if (br[j] == 0xffffffffu) continue;
        const int e = lane * kChunk + ((j + rot) & (kChunk - 1));
        perm[hist[br[j] >> 16] + (int)(br[j] & 0xffffu)] = (uint16_t)e;
      }
      __syncwarp();

      // the lane's kChunk consecutive positions of the sorted order
#pragma unroll 1
      for (int j = 0; j < kChunk; ++j) {
        const int pos = lane * kChunk + ((j + rot) & (kChunk - 1));
        if (pos >= nion) continue;
        const int e = perm[pos];
        int vox = TC[SL::CELL][e];
        float ox = T[SL::OX][e], oy = 0.f, oz = T[SL::OZ][e];
        float vx = T[SL::VX][e], vy = T[SL::VY][e], vz = T[SL::VZ][e];
        const float w = T[SL::W][e];
        const int own = vox;
        float cv[NV];
        const int pk = push_ion<DIM, SHAPE, MODE>(a, eb, i0, j0, k0, vox, ox, oy, oz, vx, vy,
                                                  vz, w, cv, rk);
        if (pk == INT_MIN) continue;
        if (MODE == 0) {
          TC[SL::CELL][e] = vox;
          T[SL::OX][e] = ox;
          T[SL::OZ][e] = oz;
          T[SL::VX][e] = vx;
          T[SL::VY][e] = vy;
          T[SL::VZ][e] = vz;
        }
        run.add(a, pk, own, cv);
      }
    } else {
      // quads of the memory order; lanes start at a rotated quad so that the
      // 128-bit shared loads of a quarter-warp hit distinct banks
      const int rot = CQ > 1 ? (lane / (32 / kChunk)) % CQ : 0;
#pragma unroll 1
      for (int jj = 0; jj < CQ; ++jj) {
        const int jq = (jj + rot) % CQ;
        const int lq = lane * CQ + jq;  // quad within the staging tile
        if (lq >= nqt) continue;
        const int e0 = lq * 4;
        const int4 c4 = *reinterpret_cast<const int4 *>(&TC[SL::CELL][e0]);
        int cc[4] = {c4.x, c4.y, c4.z, c4.w};
        const float4 X = *reinterpret_cast<const float4 *>(&T[SL::OX][e0]);
        const float4 Z = *reinterpret_cast<const float4 *>(&T[SL::OZ][e0]);
        float4 Y = make_float4(0.f, 0.f, 0.f, 0.f);
        if (DIM == 3) Y = *reinterpret_cast<const float4 *>(&T[SL::OY][e0]);
        const float4 VX = *reinterpret_cast<const float4 *>(&T[SL::VX][e0]);
        const float4 VY = *reinterpret_cast<const float4 *>(&T[SL::VY][e0]);
        const float4 VZ = *reinterpret_cast<const float4 *>(&T[SL::VZ][e0]);
        const float4 Wq = *reinterpret_cast<const float4 *>(&T[SL::W][e0]);
        float ox[4] = {X.x, X.y, X.z, X.w}, oy[4] = {Y.x, Y.y, Y.z, Y.w},
              oz[4] = {Z.x, Z.y, Z.z, Z.w};
        float vx[4] = {VX.x, VX.y, VX.z, VX.w}, vy[4] = {VY.x, VY.y, VY.z, VY.w},
              vz[4] = {VZ.x, VZ.y, VZ.z, VZ.w};
        const float ww[4] = {Wq.x, Wq.y, Wq.z, Wq.w};
        const int64_t ion0 = (q0 + lq) * 4;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          if (ion0 + p >= a.n) continue;
          const int own = cc[p];
          float cv[NV];
          const int pk = push_ion<DIM, SHAPE, MODE>(a, eb, i0, j0, k0, cc[p], ox[p], oy[p],
                                                    oz[p], vx[p], vy[p], vz[p], ww[p], cv, rk);
          if (pk == INT_MIN) continue;
          run.add(a, pk, own, cv);
        }
        if (MODE == 0) {
          *reinterpret_cast<int4 *>(&TC[SL::CELL][e0]) = make_int4(cc[0], cc[1], cc[2], cc[3]);
          *reinterpret_cast<float4 *>(&T[SL::OX][e0]) = make_float4(ox[0], ox[1], ox[2], ox[3]);
          if (DIM == 3)
            *reinterpret_cast<float4 *>(&T[SL::OY][e0]) = make_float4(oy[0], oy[1], oy[2], oy[3]);
          *reinterpret_cast<float4 *>(&T[SL::OZ][e0]) = make_float4(oz[0], oz[1], oz[2], oz[3]);
          *reinterpret_cast<float4 *>(&T[SL::VX][e0]) = make_float4(vx[0], vx[1], vx[2], vx[3]);
          *reinterpret_cast<float4 *>(&T[SL::VY][e0]) = make_float4(vy[0], vy[1], vy[2], vy[3]);
          *reinterpret_cast<float4 *>(&T[SL::VZ][e0]) = make_float4(vz[0], vz[1], vz[2], vz[3]);
        }
      }
    }
    run.finish(a);
    if (MODE == 0) {
#pragma unroll
      for (int m = 0; m < 4; ++m) kahan_add(ks[m], kc[m], rk[m]);
    }

    // make the staged results visible to the bulk copy and write back every
    // field but w
    fence_async_smem();
    __syncwarp();
    if (MODE == 0 && lane == 0) {
      const uint32_t bytes = (uint32_t)nqt * 16u;
#pragma unroll
      for (int f = 0; f < NA; ++f)
        if (f != SL::W) bulk_store(reinterpret_cast<char *>(gp[f]) + q0 * 16, T[f], bytes);
      bulk_commit();
    }
  }
  if (failed && lane == 0) atomicOr(a.err, kErrTimeout);
  if (lane == 0) bulk_wait_all();  // stores done before the block exits
  __syncthreads();

  if (MODE == 0) {
    // FP64 block partials of W_K and P (deterministic order)
    __shared__ double red[nwarps][4];
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
size_t push_smem() {
  return Layout<DIM, SHAPE>::bytes;
}

template <int DIM, int SHAPE, int MODE>
cudaError_t launch_t(const PushArgs &a, int blocks, cudaStream_t s) {
  const size_t smem = push_smem<DIM, SHAPE, MODE>();
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(push_kernel<DIM, SHAPE, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  push_kernel<DIM, SHAPE, MODE><<<blocks, kThreads, smem, s>>>(a);
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

bool uses_records(const hv_ctx *c) { return c->p.shape == 1 && c->g.dim2; }


cudaError_t launch_push(hv_ctx *c, int species, int mode) {
  Species &sp = c->sp[species];
  if (sp.n == 0) return cudaSuccess;
  PushArgs a;
  a.s = sp.buf[sp.cur];
  a.n = sp.n;
  a.tile_off = sp.tile_off;
  a.EB = c->EB;
  a.acc = c->acc;
  a.accm = c->accm[c->accpar];
  a.wrapvox = c->wrapvox;
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
  const int blocks = c->g.ntiles;  // one block per supercell tile
  if (c->g.dim2) {
    return mode == 0 ? launch_shape<2, 0>(shape, a, blocks, c->stream)
                     : launch_shape<2, 1>(shape, a, blocks, c->stream);
  }
  return mode == 0 ? launch_shape<3, 0>(shape, a, blocks, c->stream)
                   : launch_shape<3, 1>(shape, a, blocks, c->stream);
}

}  // namespace hv
