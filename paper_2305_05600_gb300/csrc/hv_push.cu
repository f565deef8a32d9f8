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
// equal deposit key, flushing a run with vector reductions; the runs are
// long because the ions are kept sorted by cell (hv_sort.cu).  For QS in the
// x-z layout the accumulated quantities are the per-cell moment sums
// s*(1, dx, dx^2, dz, dz^2) of Eq. 17's weights, so every ion of a cell
// contributes to one 80-byte record; the fold kernel applies the stencil.
// For CIC, NGP and 3D QS the per-target contributions are accumulated.
#include <climits>

#include "hv_internal.cuh"

// Threads per block, resident blocks per SM the push kernel is compiled for
// (register budget 65536 / (threads * blocks)), ions per lane per staging
// tile, and ions a lane loads with one vector access.
#ifndef HV_PUSH_THREADS
#define HV_PUSH_THREADS 128
#endif
#ifndef HV_PUSH_MIN_BLOCKS
#define HV_PUSH_MIN_BLOCKS 5
#endif
// 3D: threads per block and the resident blocks per SM the registers are
// budgeted for (3 blocks of 128 threads fit by shared memory; 2 blocks of
// 256 threads at 128 registers gave 16 warps per SM instead of 12 but the
// same push time)
#ifndef HV_PUSH_THREADS_3D
#define HV_PUSH_THREADS_3D 128
#endif
#ifndef HV_PUSH_MIN_BLOCKS_3D
#define HV_PUSH_MIN_BLOCKS_3D 2
#endif
#ifndef HV_PUSH_CHUNK
#define HV_PUSH_CHUNK 8
#endif
#ifndef HV_PUSH_GROUP
#define HV_PUSH_GROUP 2
#endif
// 1: the gather accumulates E and B in packed pairs with the f32x2 fused
// multiply-add (the same IEEE fma per lane, half the instructions)
#ifndef HV_PUSH_F32X2
#define HV_PUSH_F32X2 1
#endif

namespace hv {
namespace {

constexpr unsigned kFull = 0xffffffffu;
template <int DIM>
__host__ __device__ constexpr int threads_of() {
  return DIM == 2 ? HV_PUSH_THREADS : HV_PUSH_THREADS_3D;
}
constexpr int kChunk = HV_PUSH_CHUNK;  // consecutive ions per lane per tile
constexpr int kTile = 32 * kChunk;     // ions per warp tile
constexpr int kGroup = HV_PUSH_GROUP;  // ions a lane moves with one vector access

struct PushArgs {
  Soa s;
  int64_t n;
  const int *n_dev;     // slots in use, read on the device (open faces), or null
  const int *tile_off;  // [ntiles + 1]
  const float4 *EB;
  float4 *acc;       // per-target accumulator
  float *accm;       // per-cell moment records (QS in the x-z layout)
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

// Packed pairs of FP32 values in one 64-bit register and their fused
// multiply-add, d = a * b + c per lane (sm_100 and later).
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void upk2(uint64_t v, float &lo, float &hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// E and B gathered at a particle: sum over the stencil of weight times the
// cell's {Ex, Ey, Ez, Bx} and {By, Bz}.
struct Gather {
#if HV_PUSH_F32X2
  uint64_t e01 = 0, e2b0 = 0, b12 = 0;  // (Ex, Ey), (Ez, Bx), (By, Bz)
  __device__ __forceinline__ void add(float w, float4 f0, float2 f1) {
    const uint64_t ww = pk2(w, w);
    e01 = fma2(ww, pk2(f0.x, f0.y), e01);
    e2b0 = fma2(ww, pk2(f0.z, f0.w), e2b0);
    b12 = fma2(ww, pk2(f1.x, f1.y), b12);
  }
  __device__ __forceinline__ void get(float &ex, float &ey, float &ez, float &bx, float &by,
                                      float &bz) const {
    upk2(e01, ex, ey);
    upk2(e2b0, ez, bx);
    upk2(b12, by, bz);
  }
#else
  float ex = 0.f, ey = 0.f, ez = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
  __device__ __forceinline__ void add(float w, float4 f0, float2 f1) {
    ex = fmaf(w, f0.x, ex);
    ey = fmaf(w, f0.y, ey);
    ez = fmaf(w, f0.z, ez);
    bx = fmaf(w, f0.w, bx);
    by = fmaf(w, f1.x, by);
    bz = fmaf(w, f1.y, bz);
  }
  __device__ __forceinline__ void get(float &ex_, float &ey_, float &ez_, float &bx_, float &by_,
                                      float &bz_) const {
    ex_ = ex; ey_ = ey; ez_ = ez; bx_ = bx; by_ = by; bz_ = bz;
  }
#endif
};

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

// Deposit of one ion in factored form: its NV values are the products
// f[i] * sv[c] of the factors f and sv = s * (1, vx, vy, vz), s = q w / V_c.
// QS x-z records: f = (1, dx, dx^2, dz, dz^2), value 5c + i (moment sums);
// other shapes: f = the target weights, value 4i + c.  Returns the voxel
// shift of the deposit key.
template <int DIM, int SHAPE>
struct Dep {
  static constexpr int NF = Shape<DIM, SHAPE>::REC ? 5 : Shape<DIM, SHAPE>::NT;
  float f[NF];
  float sv[4];
  __device__ __forceinline__ float value(int j) const {
    return Shape<DIM, SHAPE>::REC ? f[j % 5] * sv[j / 5] : f[j / 4] * sv[j % 4];
  }
  __device__ __forceinline__ float fma_into(int j, float acc) const {
    return Shape<DIM, SHAPE>::REC ? fmaf(f[j % 5], sv[j / 5], acc) : fmaf(f[j / 4], sv[j % 4], acc);
  }
};

template <int DIM, int SHAPE>
__device__ __forceinline__ int deposit_factors(float hx, float hy, float hz, float s, float vx,
                                               float vy, float vz, const Geom &g,
                                               Dep<DIM, SHAPE> &d) {
  d.sv[0] = s;
  d.sv[1] = s * vx;
  d.sv[2] = s * vy;
  d.sv[3] = s * vz;
  if (Shape<DIM, SHAPE>::REC) {
    d.f[0] = 1.f;
    d.f[1] = hx;
    d.f[2] = hx * hx;
    d.f[3] = hz;
    d.f[4] = hz * hz;
    return 0;
  }
  return shape_weights<DIM, SHAPE>(hx, hy, hz, g, d.f);
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

static_assert(kChunk == 8 || kChunk == 16 || kChunk == 32, "chunk: 8, 16 or 32 ions per lane");
static_assert(kGroup == 4 || kGroup == 2, "ion group: 4 or 2");

constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// One window cell of E and B in shared memory.  The x-z layout keeps the
// gather array's two float4 ({Ex,Ey,Ez,Bx}, {By,Bz,-,-}); 3D packs the six
// values into three float2 so that the larger 3D window leaves room for a
// third block per SM.
template <int DIM>
struct WinCell {
  static constexpr int kBytes = DIM == 2 ? 32 : 24;
  __device__ __forceinline__ static void store(void *win, int c, float4 e0, float4 e1) {
    if (DIM == 2) {
      float4 *w = reinterpret_cast<float4 *>(win);
      w[2 * c] = e0;
      w[2 * c + 1] = e1;
    } else {
      float2 *w = reinterpret_cast<float2 *>(win);
      w[3 * c] = make_float2(e0.x, e0.y);
      w[3 * c + 1] = make_float2(e0.z, e0.w);
      w[3 * c + 2] = make_float2(e1.x, e1.y);
    }
  }
  // E and B of cell c: {Ex, Ey, Ez, Bx} and {By, Bz}
  __device__ __forceinline__ static void load(const void *win, int c, float4 &e0, float2 &e1) {
    if (DIM == 2) {
      const float4 *w = reinterpret_cast<const float4 *>(win);
      e0 = w[2 * c];
      const float4 b = w[2 * c + 1];
      e1 = make_float2(b.x, b.y);
    } else {
      const float2 *w = reinterpret_cast<const float2 *>(win);
      const float2 a = w[3 * c], b = w[3 * c + 1];
      e0 = make_float4(a.x, a.y, b.x, b.y);
      e1 = w[3 * c + 2];
    }
  }
};

// Shared-memory layout of one push block (one supercell tile).
//   stage: one kTile-ion staging buffer per warp (bulk-copied in and out)
//   eb:    E, B of the window, 2 float4 per cell
template <int DIM, int SHAPE>
struct Layout {
  static constexpr int NW = threads_of<DIM>() / 32;
  static constexpr int NA = DIM == 2 ? 7 : 8;  // cell, ox, [oy], oz, vx, vy, vz, w
  static constexpr size_t stage_bytes = (size_t)NA * kTile * 4;
  static constexpr size_t off_eb = align_up(stage_bytes * NW, 16);
  static constexpr size_t off_bar = off_eb + (size_t)Win<DIM>::NEB * WinCell<DIM>::kBytes;
  static constexpr size_t bytes = off_bar + 8 * NW;
};

// Array slot of each particle field in a staging buffer.
template <int DIM>
struct Slot {
  static constexpr int CELL = 0, OX = 1, OY = DIM == 3 ? 2 : 1, OZ = DIM == 3 ? 3 : 2,
                       VX = OZ + 1, VY = OZ + 2, VZ = OZ + 3, W = OZ + 4;
};

// kGroup consecutive 32-bit values of a staging array (128- or 64-bit
// shared accesses).
template <int G, class E>
__device__ __forceinline__ void ldv(const E *src, E *out) {
  static_assert(sizeof(E) == 4 && (G == 4 || G == 2), "4 or 2 values of 32 bits");
  if constexpr (G == 4) {
    const uint4 v = *reinterpret_cast<const uint4 *>(src);
    const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) out[i] = __builtin_bit_cast(E, u[i]);
  } else {
    const uint2 v = *reinterpret_cast<const uint2 *>(src);
    out[0] = __builtin_bit_cast(E, v.x);
    out[1] = __builtin_bit_cast(E, v.y);
  }
}

template <int G, class E>
__device__ __forceinline__ void stv(E *dst, const E *in) {
  if constexpr (G == 4) {
    *reinterpret_cast<uint4 *>(dst) =
        make_uint4(__builtin_bit_cast(uint32_t, in[0]), __builtin_bit_cast(uint32_t, in[1]),
                   __builtin_bit_cast(uint32_t, in[2]), __builtin_bit_cast(uint32_t, in[3]));
  } else {
    *reinterpret_cast<uint2 *>(dst) =
        make_uint2(__builtin_bit_cast(uint32_t, in[0]), __builtin_bit_cast(uint32_t, in[1]));
  }
}

// Global array of staging slot f (f is a compile-time constant at every
// use, so no pointer is held in registers).
template <int DIM>
__device__ __forceinline__ char *field_ptr(const Soa &s, int f) {
  using SL = Slot<DIM>;
  if (f == SL::CELL) return reinterpret_cast<char *>(s.cell);
  if (f == SL::OX) return reinterpret_cast<char *>(s.ox);
  if (DIM == 3 && f == SL::OY) return reinterpret_cast<char *>(s.oy);
  if (f == SL::OZ) return reinterpret_cast<char *>(s.oz);
  if (f == SL::VX) return reinterpret_cast<char *>(s.vx);
  if (f == SL::VY) return reinterpret_cast<char *>(s.vy);
  if (f == SL::VZ) return reinterpret_cast<char *>(s.vz);
  return reinterpret_cast<char *>(s.w);
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

// One ion of the step: gather E^n, B^n at x^n, Boris push, move to x^{n+1}
// (MODE 0 and 2; the state is updated in place and the kinetic-energy/
// momentum terms are added to rk), then the deposit values at the half-step
// position.  MODE 2 and 3 are relativistic: the state carries u = gamma v,
// the Boris rotation uses (q dt / 2m) B / gamma^-, positions and currents
// use v = u / gamma, and the kinetic energy is m w |u|^2 / (gamma + 1).  Returns the voxel of the deposit key, or INT_MIN for a corrupt
// cell index (latched in the error word; the ion is left as it is).
template <int DIM, int SHAPE, int MODE>
__device__ __forceinline__ int push_ion(const PushArgs &a, const void *eb, int i0, int j0,
                                        int k0, int &vox, float &ox, float &oy, float &oz,
                                        float &vx, float &vy, float &vz, float w,
                                        Dep<DIM, SHAPE> &dep, float *rk) {
  using W = Win<DIM>;
  constexpr int NT = Shape<DIM, SHAPE>::NT;
  const Geom &g = a.g;
  const int vox0 = vox;
  if (vox0 == kDeadVox) return INT_MIN;  // left through an open face earlier
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
  constexpr bool PUSH = (MODE & 1) == 0, REL = MODE >= 2;
  const float dy0 = DIM == 3 ? oy : 0.f;
  float vxp = vx, vyp = vy, vzp = vz;
  float hx = ox, hy = dy0, hz = oz;
  int shx = 0, shy = 0, shz = 0;

  if (PUSH) {
    // gather E^n, B^n at x^n with the deposit's weights (App. B)
    float wt[NT];
    const int ks_ = shape_weights<DIM, SHAPE>(ox, dy0, oz, g, wt);
    Gather gat;
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
        float4 f0;
        float2 f1;
        WinCell<DIM>::load(eb, eb0 + wo, f0, f1);
        gat.add(wt[t], f0, f1);
      }
    } else {
      const int pc = vox0 + ks_;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const int pt = pc + target_off<DIM, SHAPE>(t, g);
        const float4 f0 = __ldg(a.EB + 2 * pt);
        const float4 f1 = __ldg(a.EB + 2 * pt + 1);
        gat.add(wt[t], f0, make_float2(f1.x, f1.y));
      }
    }
    float ex, ey, ez, bx, by, bz;
    gat.get(ex, ey, ez, bx, by, bz);
    // Boris: half E kick, rotation, half E kick (Eq. 9)
    const float h = a.k.qmdt2;
    const float vmx = vxp + h * ex, vmy = vyp + h * ey, vmz = vzp + h * ez;
    float tx = h * bx, ty = h * by, tz = h * bz;
    if (REL) {  // rotation of u^- by (q dt / 2m) B / gamma^-
      const float ig = __frcp_rn(sqrtf(1.f + (vmx * vmx + vmy * vmy + vmz * vmz) * a.k.ic2));
      tx *= ig;
      ty *= ig;
      tz *= ig;
    }
    // 2 / (1 + |t|^2) by the fast approximate division: the divisor is at
    // least 1, where its error stays within 2 ulp
    const float f = __fdividef(2.f, 1.f + (tx * tx + ty * ty + tz * tz));
    const float sx = f * tx, sy = f * ty, sz = f * tz;
    const float vpx = vmx + (vmy * tz - vmz * ty);
    const float vpy = vmy + (vmz * tx - vmx * tz);
    const float vpz = vmz + (vmx * ty - vmy * tx);
    vxp = vmx + (vpy * sz - vpz * sy) + h * ex;
    vyp = vmy + (vpz * sx - vpx * sz) + h * ey;
    vzp = vmz + (vpx * sy - vpy * sx) + h * ez;
    // the new state (u for the relativistic push) and the velocity that
    // moves and deposits
    float unx = vxp, uny = vyp, unz = vzp, gam = 1.f;
    if (REL) {
      gam = sqrtf(1.f + (unx * unx + uny * uny + unz * unz) * a.k.ic2);
      const float ig = __frcp_rn(gam);
      vxp = unx * ig;
      vyp = uny * ig;
      vzp = unz * ig;
    }

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
      vxp = unx = vx;
      vyp = uny = vy;
      vzp = unz = vz;
    }
    shx = rebase(hx);
    shz = rebase(hz);
    const int mx = rebase(nxo), mz = rebase(nzo);
    int my = 0;
    if (DIM == 3) {
      shy = rebase(hy);
      my = rebase(nyo);
    }
    // new cell, wrapped into the interior (periodic), or the ion leaves
    // through an open face (Sec. 2.3) and its slot is marked dead
    const int i1 = ip - kGhost + mx, k1 = kp - kGhost + mz;
    const int j1 = DIM == 2 ? 0 : jp - kGhost + my;
    const int iw = i1 < 0 ? i1 + g.nx : (i1 >= g.nx ? i1 - g.nx : i1);
    const int kw = k1 < 0 ? k1 + g.nz : (k1 >= g.nz ? k1 - g.nz : k1);
    const int jw = DIM == 2 ? 0 : (j1 < 0 ? j1 + g.ny : (j1 >= g.ny ? j1 - g.ny : j1));
    vox = voxel_of(g, iw, jw, kw);
    if (g.any_open && ((g.open[0] && iw != i1) || (g.open[2] && kw != k1) ||
                       (DIM == 3 && g.open[1] && jw != j1)))
      vox = kDeadVox;
    ox = nxo;
    if (DIM == 3) oy = nyo;
    oz = nzo;
    vx = unx;
    vy = uny;
    vz = unz;
    // w |u|^2 (over gamma + 1) and w u; the species mass (and the 1/2 of
    // the non-relativistic energy) is applied to the FP64 block sums
    const float uu = unx * unx + uny * uny + unz * unz;
    rk[0] = REL ? fmaf(w * uu, __frcp_rn(gam + 1.f), rk[0]) : fmaf(w, uu, rk[0]);
    rk[1] = fmaf(w, unx, rk[1]);
    rk[2] = fmaf(w, uny, rk[2]);
    rk[3] = fmaf(w, unz, rk[3]);
  } else if (REL) {
    // start-up deposit of a relativistic particle: v = u / gamma
    const float ig = __frcp_rn(sqrtf(1.f + (vx * vx + vy * vy + vz * vz) * a.k.ic2));
    vxp = vx * ig;
    vyp = vy * ig;
    vzp = vz * ig;
  }

  // deposit q w S / V_c and q w v S / V_c at the half-step position
  const int kshift = deposit_factors<DIM, SHAPE>(hx, hy, hz, a.k.qvc * w, vxp, vyp, vzp, g, dep);
  return vox0 + shx + shz * g.sz + (DIM == 3 ? shy * g.sy : 0) + kshift;
}

// A lane's register run: the deposit values summed over consecutive ions
// with the same deposit key.  An ion with another key flushes the run and
// starts a new one.  (Keeping the run across a single ion that left its
// cell saves a flush, but the third branch it needs makes the warp issue
// all three paths on almost every ion.)
template <int DIM, int SHAPE>
struct Run {
  static constexpr int NV = Shape<DIM, SHAPE>::NV;
  int key;
  float acc[NV];

  __device__ __forceinline__ void reset() {
    key = INT_MIN;
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = 0.f;
  }
  __device__ __forceinline__ void add(const PushArgs &a, int pk, const Dep<DIM, SHAPE> &d) {
    if (pk != key) {
      if (key != INT_MIN) flush_direct<DIM, SHAPE>(a, key, acc);
      key = pk;
#pragma unroll
      for (int j = 0; j < NV; ++j) acc[j] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = d.fma_into(j, acc[j]);
  }
  // End of a staging tile, called by all 32 lanes: lanes whose open runs
  // share a key (neighbouring lanes of a sorted tile) sum them with a
  // segmented shuffle reduction, and one lane per key flushes.
  __device__ __forceinline__ void finish(const PushArgs &a) {
    const int lane = threadIdx.x & 31;
    const int knext = __shfl_down_sync(kFull, key, 1);
    const int kprev = __shfl_up_sync(kFull, key, 1);
    bool cut = lane == 31 || knext != key;  // a segment ends at this lane
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      if (__all_sync(kFull, cut)) break;  // every segment is closed: nothing left to combine
      const bool cut_o = __shfl_down_sync(kFull, cut, o);
      const bool take = !cut && lane + o < 32;
#pragma unroll
      for (int j = 0; j < NV; ++j) {
        const float v = __shfl_down_sync(kFull, acc[j], o);
        if (take) acc[j] += v;
      }
      cut = cut || cut_o;
    }
    const bool head = lane == 0 || kprev != key;
    if (head && key != INT_MIN) flush_direct<DIM, SHAPE>(a, key, acc);
    key = INT_MIN;
  }
};


// MODE 0: full step.  MODE 1: start-up deposit at the current position with
// the stored velocity (no push, no move, no write-back).  MODE 2 and 3: the
// same with the relativistic push.
//
// kPushSplit blocks per supercell tile, each taking a contiguous part of the
// tile's ion range (finer work units than whole tiles keep the last wave of
// blocks short).  Ions are kept sorted tile-major, so the tile's ion range
// [tile_off[t], tile_off[t+1]) (rounded to whole quads) lies in the tile,
// give or take the drift since the last sort.  The block stages E and B of
// the tile and a halo in shared memory; ions that drifted further gather
// from global memory.  Each warp streams tiles of kTile ions
// through shared memory with bulk copies; each lane takes kChunk consecutive
// ions and sums their deposits in registers per run of equal deposit key,
// flushing a run with vector reductions into the global accumulator.  The
// staging tile is written back in place with bulk copies.
template <int DIM, int SHAPE, int MODE>
// (3D: the larger staging and window buffers allow two blocks per SM)
__global__ void __launch_bounds__(threads_of<DIM>(),
                                  DIM == 2 ? HV_PUSH_MIN_BLOCKS : HV_PUSH_MIN_BLOCKS_3D)
    push_kernel(PushArgs a) {
  pdl_begin();
  constexpr bool PUSH = (MODE & 1) == 0;  // full step (not the start-up deposit)
  using L = Layout<DIM, SHAPE>;
  using W = Win<DIM>;
  using SL = Slot<DIM>;
  constexpr int NA = L::NA;
  constexpr int CG = kChunk / kGroup;  // ion groups per lane per staging tile
  constexpr int TQ = kTile / 4;        // quads per staging tile
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const Geom &g = a.g;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int kThreads = threads_of<DIM>();
  constexpr int nwarps = kThreads / 32;
  float(&T)[NA][kTile] = *reinterpret_cast<float(*)[NA][kTile]>(smem_raw + L::stage_bytes * warp);
  int(&TC)[NA][kTile] = *reinterpret_cast<int(*)[NA][kTile]>(smem_raw + L::stage_bytes * warp);
  void *eb = smem_raw + L::off_eb;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + L::off_bar) + warp;

  // tile origin and the block's range of quads: kPushSplit blocks share a
  // tile, each taking a contiguous part of its staging tiles
  const int tile = blockIdx.x / kPushSplit;
  const int part = blockIdx.x % kPushSplit;
  const int ti = tile % g.ntx, tj = (tile / g.ntx) % g.nty, tk = tile / (g.ntx * g.nty);
  const int i0 = ti * W::TX, j0 = tj * W::TY, k0 = tk * W::TZ;
  const int64_t n_ions = a.n_dev ? (int64_t)*a.n_dev : a.n;
  const int64_t nq = (n_ions + 3) >> 2;
  const int64_t qa = tile == 0 ? 0 : (int64_t)a.tile_off[tile] >> 2;
  const int64_t qe = tile == g.ntiles - 1 ? nq : (int64_t)a.tile_off[tile + 1] >> 2;
  const int64_t nst = qe > qa ? (qe - qa + TQ - 1) / TQ : 0;  // staging tiles of the tile
  const int64_t st_lo = nst * part / kPushSplit, st_hi = nst * (part + 1) / kPushSplit;

  // bulk loads of staging tile st into the warp's buffer
  auto issue = [&](int64_t st) {
    const int64_t q0 = qa + st * TQ;
    const uint32_t bytes = (uint32_t)min((int64_t)TQ, qe - q0) * 16u;
    mbar_expect_tx(bar, bytes * NA);
#pragma unroll
    for (int f = 0; f < NA; ++f) bulk_load(T[f], field_ptr<DIM>(a.s, f) + q0 * 16, bytes, bar);
  };
  // the warp's first staging tile is requested before the window is staged,
  // so that the two loads overlap
  if (lane == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (st_lo + warp < st_hi) issue(st_lo + warp);
  }

  // stage E, B of the window
  if (PUSH) {
    for (int c = threadIdx.x; c < W::NEB; c += kThreads) {
      const int wx = c % W::EX, wy = (c / W::EX) % W::EY, wz = c / (W::EX * W::EY);
      const int ip = i0 + wx - W::RE + kGhost, kp = k0 + wz - W::RE + kGhost;
      const int jp = DIM == 2 ? 0 : j0 + wy - W::RE + kGhost;
      if (ip < 0 || ip >= g.px || kp < 0 || kp >= g.pz || (DIM == 3 && (jp < 0 || jp >= g.py)))
        continue;  // outside the padded grid: never read by an in-window ion
      const int v = ip + (DIM == 2 ? 0 : jp * g.sy) + kp * g.sz;
      WinCell<DIM>::store(eb, c, __ldg(a.EB + 2 * v), __ldg(a.EB + 2 * v + 1));
    }
  }
  __syncthreads();

  float ks[4] = {0.f, 0.f, 0.f, 0.f}, kc[4] = {0.f, 0.f, 0.f, 0.f};
  bool failed = false;
  int k = 0;

  for (int64_t st = st_lo + warp; st < st_hi && !failed; st += nwarps, ++k) {
    const int64_t q0 = qa + st * TQ;
    const int nqt = (int)min((int64_t)TQ, qe - q0);
    if (lane == 0 && k > 0) {
      bulk_wait_read_all();  // the previous store has read the buffer
      issue(st);
    }
    // the warp gives up together if any lane's bounded wait ran out
    if (__any_sync(kFull, !mbar_wait_bounded(bar, (uint32_t)(k & 1)))) {
      failed = true;
      mbar_wait_bounded(bar, (uint32_t)(k & 1));  // one more bounded chance
      break;
    }

    Run<DIM, SHAPE> run;
    run.reset();
    float rk[4] = {0.f, 0.f, 0.f, 0.f};

    // groups of kGroup ions of the memory order; lanes start at a rotated
    // group so that the vector shared loads of a phase hit distinct banks
    const int rot = CG > 1 ? (lane / (32 / kChunk)) % CG : 0;
#pragma unroll 1
    for (int jj = 0; jj < CG; ++jj) {
      const int lg = lane * CG + (jj + rot) % CG;  // group within the staging tile
      const int e0 = lg * kGroup;
      if (e0 >= nqt * 4) continue;
      int cc[kGroup];
      float ox[kGroup], oy[kGroup], oz[kGroup], vx[kGroup], vy[kGroup], vz[kGroup], ww[kGroup];
      ldv<kGroup>(&TC[SL::CELL][e0], cc);
      ldv<kGroup>(&T[SL::OX][e0], ox);
      if (DIM == 3) ldv<kGroup>(&T[SL::OY][e0], oy);
      ldv<kGroup>(&T[SL::OZ][e0], oz);
      ldv<kGroup>(&T[SL::VX][e0], vx);
      ldv<kGroup>(&T[SL::VY][e0], vy);
      ldv<kGroup>(&T[SL::VZ][e0], vz);
      ldv<kGroup>(&T[SL::W][e0], ww);
      const int64_t nvalid = n_ions - (q0 * 4 + e0);  // ions of the group that exist
#pragma unroll
      for (int p = 0; p < kGroup; ++p) {
        if (p >= nvalid) continue;
        Dep<DIM, SHAPE> dep;
        const int pk = push_ion<DIM, SHAPE, MODE>(a, eb, i0, j0, k0, cc[p], ox[p], oy[p], oz[p],
                                                  vx[p], vy[p], vz[p], ww[p], dep, rk);
        if (pk == INT_MIN) continue;
        run.add(a, pk, dep);
      }
      if (PUSH) {
        stv<kGroup>(&TC[SL::CELL][e0], cc);
        stv<kGroup>(&T[SL::OX][e0], ox);
        if (DIM == 3) stv<kGroup>(&T[SL::OY][e0], oy);
        stv<kGroup>(&T[SL::OZ][e0], oz);
        stv<kGroup>(&T[SL::VX][e0], vx);
        stv<kGroup>(&T[SL::VY][e0], vy);
        stv<kGroup>(&T[SL::VZ][e0], vz);
      }
    }
    run.finish(a);
    if (PUSH) {
#pragma unroll
      for (int m = 0; m < 4; ++m) kahan_add(ks[m], kc[m], rk[m]);
    }

    // make the staged results visible to the bulk copy and write back every
    // field but w
    fence_async_smem();
    __syncwarp();
    if (PUSH && lane == 0) {
      const uint32_t bytes = (uint32_t)nqt * 16u;
#pragma unroll
      for (int f = 0; f < NA; ++f)
        if (f != SL::W) bulk_store(field_ptr<DIM>(a.s, f) + q0 * 16, T[f], bytes);
      bulk_commit();
    }
  }
  if (failed && lane == 0) atomicOr(a.err, kErrTimeout);
  if (lane == 0) bulk_wait_all();  // stores done before the block exits
  __syncthreads();

  if (PUSH) {
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
      const double m = a.k.mass_d;
      a.part[(int64_t)blockIdx.x * 4 + threadIdx.x] =
          s * (threadIdx.x == 0 && MODE < 2 ? 0.5 * m : m);
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
  static std::atomic<uint64_t> attr_set{0};
  cudaError_t e = set_smem_once(push_kernel<DIM, SHAPE, MODE>, smem, attr_set);
  if (e != cudaSuccess) return e;
  // an ordinary launch: the push may follow a wait on the side stream's
  // sort, which a programmatic launch must not overtake
  push_kernel<DIM, SHAPE, MODE><<<blocks, threads_of<DIM>(), smem, s>>>(a);
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
  a.n_dev = c->g.any_open ? sp.n_used : nullptr;
  a.tile_off = sp.tile_off;
  a.EB = gather_array(c);
  a.acc = c->acc;
  a.accm = c->accm[c->accpar];
  a.g = c->g;
  a.k.qmdt2 = (float)(0.5 * sp.q / sp.m * c->p.dt);
  a.k.cx = c->g.nx > 1 ? (float)(c->p.dt / c->p.dx) : 0.f;
  a.k.cy = c->g.ny > 1 ? (float)(c->p.dt / c->p.dy) : 0.f;
  a.k.cz = c->g.nz > 1 ? (float)(c->p.dt / c->p.dz) : 0.f;
  a.k.qvc = (float)(sp.q / c->vc);
  a.k.ic2 = c->p.relativistic ? (float)(1.0 / (c->p.c_light * c->p.c_light)) : 0.f;
  a.k.mass_d = sp.m;
  a.part = c->pushpart + (size_t)species * c->push_blocks * 4;
  a.err = c->err;
  c->launches++;
  const int shape = c->p.shape;
  const int blocks = c->push_blocks;  // kPushSplit blocks per supercell tile
  const int m = mode + (c->p.relativistic ? 2 : 0);
  if (c->g.dim2) {
    switch (m) {
      case 0: return launch_shape<2, 0>(shape, a, blocks, c->stream);
      case 1: return launch_shape<2, 1>(shape, a, blocks, c->stream);
      case 2: return launch_shape<2, 2>(shape, a, blocks, c->stream);
      default: return launch_shape<2, 3>(shape, a, blocks, c->stream);
    }
  }
  switch (m) {
    case 0: return launch_shape<3, 0>(shape, a, blocks, c->stream);
    case 1: return launch_shape<3, 1>(shape, a, blocks, c->stream);
    case 2: return launch_shape<3, 2>(shape, a, blocks, c->stream);
    default: return launch_shape<3, 3>(shape, a, blocks, c->stream);
  }
}

}  // namespace hv
