// Grid kernels of the hybrid PIC step on the cell-centred grid (Sec. 2.2):
//  * moment post: fold the ghost layer of the deposit accumulator back onto
//    the periodic interior, optional binomial smoothing, linear
//    extrapolation (Eq. 11);
//  * field stage: one fused explicit-midpoint stage of the subcycled
//    Faraday update (Eq. 5) with E from Ohm's law (Eqs. 2-4, 6) and the
//    density floor, computed tile by tile in shared memory (halo 3: J = curl B
//    needs B at +-1, the hyper-resistive Laplacian needs J at +-1, and curl E
//    needs E at +-1);
//  * final Ohm: E^{n+1} written with B^{n+1} into the ghost-padded gather
//    array;
//  * diagnostics: FP64 block partials of sum |B|^2/2 V_c, sum n V_c and
//    max |div B|, reduced in a fixed order with the particle partials.
#include <algorithm>
#include <utility>

#include "hv_internal.cuh"

namespace hv {
namespace {

__device__ __forceinline__ int wrapn(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Periodic wrap of a coordinate at most `h` cells outside [0, n): two
// compares instead of a division when n >= h.
__device__ __forceinline__ int wrap_near(int i, int n, int h) {
  if (n >= h) return i < 0 ? i + n : (i >= n ? i - n : i);
  return wrapn(i, n);
}

__device__ __forceinline__ void decode(const Geom &g, int c, int &i, int &j, int &k) {
  const int q = (int)fdiv((uint32_t)c, g.div_nx);
  i = c - q * g.nx;
  k = (int)fdiv((uint32_t)q, g.div_ny);
  j = q - k * g.ny;
}

struct MomArgs {
  Geom g;
  float4 *acc;            // per-target accumulator (read and zeroed)
  const float *rec;       // moment records of this step (read)
  const float4 *prev_in;  // n^{n-1/2}, J^{n-1/2}
  float4 *raw_out;        // folded deposit (when smoothing follows)
  float4 *prev_out;       // n^{n+1/2}, J^{n+1/2}
  float4 *ext_out;        // extrapolated n^{n+1}, J^{n+1}
  int fuse;               // 1: fold + extrapolate in one pass
  int init;               // 1: start-up (prev := ext := deposit)
};

__device__ __forceinline__ void finish_moment(const MomArgs &a, int c, float4 m) {
  if (!a.fuse) {
    a.raw_out[c] = m;
    return;
  }
  if (a.init) {
    a.prev_out[c] = m;
    a.ext_out[c] = m;
    return;
  }
  const float4 pv = a.prev_in[c];
  a.ext_out[c] = make_float4(1.5f * m.x - 0.5f * pv.x, 1.5f * m.y - 0.5f * pv.y,
                             1.5f * m.z - 0.5f * pv.z, 1.5f * m.w - 0.5f * pv.w);
  a.prev_out[c] = m;
}

// Fold the per-target accumulator onto the periodic interior: every padded
// voxel that stands for the cell (the cell and its ghost images) is summed;
// then (fused) extrapolate with Eq. 11.  The accumulator is cleared for the
// next step by a memset after the fold: zeroing each voxel right after
// reading it made the 3D fold six times slower on GB300.
__global__ void __launch_bounds__(256) fold_kernel(MomArgs a) {
  pdl_begin();
  const Geom &g = a.g;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, c, i, j, k);
    float4 m = make_float4(0.f, 0.f, 0.f, 0.f);
    if (single_image(g, i, j, k)) {
      const int p = voxel_of(g, i, j, k);
      const float4 v = a.acc[p];
      m.x += v.x;
      m.y += v.y;
      m.z += v.z;
      m.w += v.w;
      finish_moment(a, c, m);
      continue;
    }
    int xs[5], ys[5], zs[5];
    const int nxs = axis_sources(i, g.nx, g.open[0], xs);
    const int nys = g.dim2 ? 1 : axis_sources(j, g.ny, g.open[1], ys);
    if (g.dim2) ys[0] = 0;
    const int nzs = axis_sources(k, g.nz, g.open[2], zs);
    for (int a3 = 0; a3 < nzs; ++a3)
      for (int a2 = 0; a2 < nys; ++a2)
        for (int a1 = 0; a1 < nxs; ++a1) {
          const int p = xs[a1] + ys[a2] * g.sy + zs[a3] * g.sz;
          const float4 v = a.acc[p];
          m.x += v.x;
          m.y += v.y;
          m.z += v.z;
          m.w += v.w;
        }
    finish_moment(a, c, m);
  }
}

// Fold of the QS moment records (x-z layout): a record holds, per channel,
// the sums S0, Sx, Sxx, Sz, Szz of s, s dx, s dx^2, s dz, s dz^2 over the ions
// whose half-step cell is that voxel.  Eq. 17 gives the voxel itself
// (4 S0 - Sxx - Szz)/6 (the two y neighbours of the single y cell folded in),
// its x+-1 neighbours (S0 +- 2 Sx + Sxx)/12 and its z+-1 neighbours
// (S0 +- 2 Sz + Szz)/12.  A cell collects from every source voxel whose
// stencil reaches one of its images.  (The buffer read here is cleared
// for its next deposit by the host, beside the field advance.)
__global__ void __launch_bounds__(256) fold_records_kernel(MomArgs a) {
  pdl_begin();
  const Geom &g = a.g;
  const float c6 = 1.f / 6.f, c12 = 1.f / 12.f;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, c, i, j, k);
    int xs[5], zs[5];
    const int nxs = axis_sources(i, g.nx, g.open[0], xs);
    const int nzs = axis_sources(k, g.nz, g.open[2], zs);
    float m[4] = {0.f, 0.f, 0.f, 0.f};
    for (int a3 = 0; a3 < nzs; ++a3)
      for (int a1 = 0; a1 < nxs; ++a1) {
        const int Px = xs[a1], Pz = zs[a3];
        const int T = Px + Pz * g.sz;
        // (dx, dz) of the target relative to the source: 0, +x, -x, +z, -z
        for (int t = 0; t < 5; ++t) {
          const int sx = t == 1 ? -1 : (t == 2 ? 1 : 0);
          const int sz = t == 3 ? -1 : (t == 4 ? 1 : 0);
          const int Qx = Px + sx, Qz = Pz + sz;
          if (Qx < 0 || Qx >= g.px || Qz < 0 || Qz >= g.pz) continue;
          const float4 *r4 = reinterpret_cast<const float4 *>(a.rec + (size_t)(Qx + Qz * g.sz) * kMono);
          const float4 q0 = r4[0], q1 = r4[1], q2 = r4[2], q3 = r4[3], q4 = r4[4];
          const float r[kMono] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y,
                                  q2.z, q2.w, q3.x, q3.y, q3.z, q3.w, q4.x, q4.y, q4.z, q4.w};
#pragma unroll
          for (int ch = 0; ch < 4; ++ch) {
            const float S0 = r[5 * ch], Sx = r[5 * ch + 1], Sxx = r[5 * ch + 2],
                        Sz = r[5 * ch + 3], Szz = r[5 * ch + 4];
            float w;
            if (t == 0) w = (4.f * S0 - Sxx - Szz) * c6;
            else if (t == 1) w = (S0 + 2.f * Sx + Sxx) * c12;
            else if (t == 2) w = (S0 - 2.f * Sx + Sxx) * c12;
            else if (t == 3) w = (S0 + 2.f * Sz + Szz) * c12;
            else w = (S0 - 2.f * Sz + Szz) * c12;
            m[ch] += w;
          }
        }
      }
    finish_moment(a, c, make_float4(m[0], m[1], m[2], m[3]));
  }
}

// One pass of the separable (1/4, 1/2, 1/4) binomial filter along every
// axis with more than one cell (tensor-product stencil), periodic.
__global__ void __launch_bounds__(256) smooth_kernel(Geom g, const float4 *in, float4 *out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, c, i, j, k);
    const float wts[3] = {0.25f, 0.5f, 0.25f};
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int dz = -1; dz <= 1; ++dz) {
      const int kk = wrapn(k + dz, g.nz);
      for (int dy = -1; dy <= 1; ++dy) {
        const int jj = wrapn(j + dy, g.ny);
        for (int dx = -1; dx <= 1; ++dx) {
          const int ii = wrapn(i + dx, g.nx);
          const float w = wts[dx + 1] * wts[dy + 1] * wts[dz + 1];
          const float4 v = in[ii + g.nx * (jj + g.ny * kk)];
          s.x = fmaf(w, v.x, s.x);
          s.y = fmaf(w, v.y, s.y);
          s.z = fmaf(w, v.z, s.z);
          s.w = fmaf(w, v.w, s.w);
        }
      }
    }
    out[c] = s;
  }
}

// Up to kSmoothMax binomial passes in one launch (x-z layout): a block
// loads a 32x32 output tile with a halo of one cell per pass into shared
// memory and applies the passes there, each on a region one cell smaller,
// as an x sweep then a z sweep of (1/4, 1/2, 1/4) (the tensor-product
// stencil of smooth_kernel, rounded per sweep).  Global memory is read and
// written once per launch instead of once per pass.
namespace smz {
constexpr int T = 32, kMax = 8, R = T + 2 * kMax, kThreads = 256;
constexpr size_t kBytes = 2 * (size_t)R * R * sizeof(float4);
}  // namespace smz

__global__ void __launch_bounds__(smz::kThreads) smooth2d_multi_kernel(Geom g, const float4 *in,
                                                                       float4 *out, int passes) {
  using namespace smz;
  extern __shared__ __align__(16) float4 sb[];
  float4 *a = sb, *b = sb + R * R;
  const int ntx = (g.nx + T - 1) / T;
  const int x0 = (blockIdx.x % ntx) * T, z0 = (blockIdx.x / ntx) * T;
  const int H = passes, W = T + 2 * H;  // loaded region W x W (row pitch R)
  for (int r = threadIdx.x; r < W * W; r += blockDim.x) {
    const int lx = r % W - H, lz = r / W - H;
    const int gx = wrapn(x0 + lx, g.nx), gz = wrapn(z0 + lz, g.nz);
    a[(lz + H) * R + (lx + H)] = in[gx + g.nx * gz];
  }
  __syncthreads();
  for (int q = 0; q < passes; ++q) {
    // region of the result of this pass: halo H - q - 1
    const int h = H - q - 1, w = T + 2 * h, o = q + 1;  // first row/column in the arrays
    // x sweep over rows o-1 .. o+w (the z sweep needs one row above and below)
    for (int r = threadIdx.x; r < w * (w + 2); r += blockDim.x) {
      const int ix = o + r % w, iz = o - 1 + r / w;
      const float4 l = a[iz * R + ix - 1], c = a[iz * R + ix], rr = a[iz * R + ix + 1];
      b[iz * R + ix] = make_float4(0.25f * l.x + 0.5f * c.x + 0.25f * rr.x,
                                   0.25f * l.y + 0.5f * c.y + 0.25f * rr.y,
                                   0.25f * l.z + 0.5f * c.z + 0.25f * rr.z,
                                   0.25f * l.w + 0.5f * c.w + 0.25f * rr.w);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < w * w; r += blockDim.x) {
      const int ix = o + r % w, iz = o + r / w;
      const float4 d = b[(iz - 1) * R + ix], c = b[iz * R + ix], u = b[(iz + 1) * R + ix];
      a[iz * R + ix] = make_float4(0.25f * d.x + 0.5f * c.x + 0.25f * u.x,
                                   0.25f * d.y + 0.5f * c.y + 0.25f * u.y,
                                   0.25f * d.z + 0.5f * c.z + 0.25f * u.z,
                                   0.25f * d.w + 0.5f * c.w + 0.25f * u.w);
    }
    __syncthreads();
  }
  for (int r = threadIdx.x; r < T * T; r += blockDim.x) {
    const int gx = x0 + r % T, gz = z0 + r / T;
    if (gx < g.nx && gz < g.nz) out[gx + g.nx * gz] = a[(r / T + H) * R + (r % T + H)];
  }
}

__global__ void __launch_bounds__(256) extrap_kernel(int ncell, const float4 *half,
                                                     const float4 *prev_in, float4 *prev_out,
                                                     float4 *ext_out, int init) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    const float4 m = half[c];
    if (init) {
      prev_out[c] = m;
      ext_out[c] = m;
      continue;
    }
    const float4 pv = prev_in[c];
    ext_out[c] = make_float4(1.5f * m.x - 0.5f * pv.x, 1.5f * m.y - 0.5f * pv.y,
                             1.5f * m.z - 0.5f * pv.z, 1.5f * m.w - 0.5f * pv.w);
    prev_out[c] = m;
  }
}

// ----------------------------------------------------------------------------
// Ohm's law + Faraday stage, tiled in shared memory
// ----------------------------------------------------------------------------

struct FieldConsts {
  float idx2, idy2, idz2;       // 1 / (2 Delta) per axis (0 on single-cell axes)
  float ilx, ily, ilz;          // 1 / Delta^2 per axis (0 on single-cell axes)
  float Te, gamma_e, eta, eta_h, n_floor;
  float kappa;                  // heat conductivity of the electron energy equation
  int model;                    // Ohm's law: 0 hybrid, 1 electrostatic, 2 resistive
  int isothermal;
};

struct StageArgs {
  Geom g;
  FieldConsts k;
  const float4 *Bin;
  const float4 *Bbase;
  float4 *Bout;
  const float4 *mom;  // {n, Jix, Jiy, Jiz}
  float coef;         // B_out = B_base - coef * curl E
  float4 *EB;         // final variant: padded gather array
  // electron energy equation (PEQ variants): p_e of the stage input, of the
  // base and the output, p_out = p_base + pcoef * dp_e/dt
  const float *pin, *pbase;
  float *pout;
  float pcoef;
  const float4 *B0;   // external field (interior) or null: B arrays hold B1
};

// Output tile and halos.  FINAL = 0: stage (E on halo 1, B on halo 3);
// FINAL = 1: E on the tile itself (B on halo 2), or with OPEN on halo 1 too
// (the ghost cells beyond open faces get their own E).  DIM = 2: x-z plane.
// PEQ: p_e is a field (electron energy equation), read instead of the
// equation of state; a stage also advances it and keeps u_e, p_e u_e and
// T_e on the E region.  OPEN: some axes have open faces (Sec. 2.3).
template <int DIM, int FINAL, int PEQ = 0, int OPEN = 0>
struct Tile {
  static constexpr int OX = DIM == 2 ? 32 : 8;
  static constexpr int OY = DIM == 2 ? 1 : 8;
  static constexpr int OZ = DIM == 2 ? 16 : 4;
  static constexpr int HE = FINAL && !OPEN ? 0 : 1;  // E halo
  static constexpr int HJ = HE + 1;         // J, n halo
  static constexpr int HB = HE + 2;         // B halo
  static constexpr int HY = DIM == 2 ? 0 : 1;  // y halos scale by this
  template <int H>
  struct R {
    static constexpr int X = OX + 2 * H, Y = OY + 2 * H * HY, Z = OZ + 2 * H;
    static constexpr int N = X * Y * Z;
  };
  static constexpr int NB = R<HB>::N, NJ = R<HJ>::N, NE = R<HE>::N;
  static constexpr int NX = PEQ && !FINAL ? 7 * NE : 0;  // u_e, p_e u_e, T_e
  static constexpr size_t smem_floats = 3 * NB + 3 * NJ + 2 * NJ + 3 * NE + NX;
};

// With OPEN (open faces, Sec. 2.3): B1, B0 and the moments beyond an open
// face are read from the interior cell next to it (clamped index), and in a
// cell beyond an open face every derivative normal to that face is zero
// (J = curl B1, the Laplacian of J, grad p_e): Ohm's law in the ghost cell
// has no normal gradients.  The final variant also writes E and B of the
// ghost cells into the first ghost layer of the gather array.
template <int DIM, int FINAL, int PEQ = 0, int OPEN = 0>
__global__ void __launch_bounds__(256) stage_kernel(StageArgs a) {
  pdl_begin();
  using T = Tile<DIM, FINAL, PEQ, OPEN>;
  using RB = typename T::template R<T::HB>;
  using RJ = typename T::template R<T::HJ>;
  using RE = typename T::template R<T::HE>;
  extern __shared__ float sm[];
  float *Bx = sm, *By = Bx + RB::N, *Bz = By + RB::N;
  float *Jx = Bz + RB::N, *Jy = Jx + RJ::N, *Jz = Jy + RJ::N;
  float *nf = Jz + RJ::N, *pe = nf + RJ::N;
  float *Ex = pe + RJ::N, *Ey = Ex + RE::N, *Ez = Ey + RE::N;
  float *Ux = Ez + RE::N, *Uy = Ux + RE::N, *Uz = Uy + RE::N;      // PEQ: u_e
  float *Px = Uz + RE::N, *Py = Px + RE::N, *Pz = Py + RE::N;      // PEQ: p_e u_e
  float *Tel = Pz + RE::N;                                         // PEQ: T_e
  const Geom &g = a.g;
  const FieldConsts &k = a.k;

  const int ntx = (g.nx + T::OX - 1) / T::OX;
  const int nty = DIM == 2 ? 1 : (g.ny + T::OY - 1) / T::OY;
  const int bid = blockIdx.x;
  const int tx = bid % ntx;
  const int ty = (bid / ntx) % nty;
  const int tz = bid / (ntx * nty);
  const int x0 = tx * T::OX, y0 = ty * T::OY, z0 = tz * T::OZ;

  // global interior index of a tile-relative coordinate (periodic, or on
  // an open axis clamped to the interior cell next to the face; tiles may
  // overhang the grid by up to one tile minus a cell, halos by HB)
  auto coord = [&](int gc, int n, int open, int reach) {
    if (OPEN && open) return gc < 0 ? 0 : (gc >= n ? n - 1 : gc);
    return wrap_near(gc, n, reach);
  };
  auto gidx = [&](int lx, int ly, int lz) {
    const int ii = coord(x0 + lx, g.nx, g.open[0], T::OX + T::HB);
    const int jj = DIM == 2 ? 0 : coord(y0 + ly, g.ny, g.open[1], T::OY + T::HB);
    const int kk = coord(z0 + lz, g.nz, g.open[2], T::OZ + T::HB);
    return ii + g.nx * (jj + g.ny * kk);
  };
  // 1 where the derivative along an axis is kept: 0 in a cell beyond an
  // open face of that axis
  auto keep = [&](int gc, int n, int open) -> float {
    return (OPEN && open && (gc < 0 || gc >= n)) ? 0.f : 1.f;
  };

  // B on the B region
  for (int r = threadIdx.x; r < RB::N; r += blockDim.x) {
    const int lx = r % RB::X - T::HB;
    const int ly = (r / RB::X) % RB::Y - T::HB * T::HY;
    const int lz = r / (RB::X * RB::Y) - T::HB;
    const float4 b = a.Bin[gidx(lx, ly, lz)];
    Bx[r] = b.x;
    By[r] = b.y;
    Bz[r] = b.z;
  }
  // floored density and electron pressure on the J region
  for (int r = threadIdx.x; r < RJ::N; r += blockDim.x) {
    const int lx = r % RJ::X - T::HJ;
    const int ly = (r / RJ::X) % RJ::Y - T::HJ * T::HY;
    const int lz = r / (RJ::X * RJ::Y) - T::HJ;
    const int gi = gidx(lx, ly, lz);
    const float n = a.mom[gi].x;
    const float f = fmaxf(n, k.n_floor);
    nf[r] = f;
    pe[r] = PEQ ? a.pin[gi] : (k.isothermal ? k.Te * f : k.Te * powf(f, k.gamma_e));
  }
  __syncthreads();

  // J = curl B (centred, Eq. 12) on the J region
  constexpr int sBy = RB::X, sBz = RB::X * RB::Y;
  for (int r = threadIdx.x; r < RJ::N; r += blockDim.x) {
    const int lx = r % RJ::X - T::HJ;
    const int ly = (r / RJ::X) % RJ::Y - T::HJ * T::HY;
    const int lz = r / (RJ::X * RJ::Y) - T::HJ;
    const int b = (lx + T::HB) + (ly + T::HB * T::HY) * sBy + (lz + T::HB) * sBz;
    const float kx = keep(x0 + lx, g.nx, g.open[0]), kz = keep(z0 + lz, g.nz, g.open[2]);
    const float ky = DIM == 2 ? 1.f : keep(y0 + ly, g.ny, g.open[1]);
    const float dBz_dy = DIM == 2 ? 0.f : ky * (Bz[b + sBy] - Bz[b - sBy]) * k.idy2;
    const float dBx_dy = DIM == 2 ? 0.f : ky * (Bx[b + sBy] - Bx[b - sBy]) * k.idy2;
    const float dBy_dz = kz * (By[b + sBz] - By[b - sBz]) * k.idz2;
    const float dBx_dz = kz * (Bx[b + sBz] - Bx[b - sBz]) * k.idz2;
    const float dBz_dx = kx * (Bz[b + 1] - Bz[b - 1]) * k.idx2;
    const float dBy_dx = kx * (By[b + 1] - By[b - 1]) * k.idx2;
    Jx[r] = dBz_dy - dBy_dz;
    Jy[r] = dBx_dz - dBz_dx;
    Jz[r] = dBy_dx - dBx_dy;
  }
  __syncthreads();

  // E = [-grad p_e + (J - J_i) x B] / n_f + eta J - eta_H lap J (Eqs. 2-4, 6)
  constexpr int sJy = RJ::X, sJz = RJ::X * RJ::Y;
  for (int r = threadIdx.x; r < RE::N; r += blockDim.x) {
    const int lx = r % RE::X - T::HE;
    const int ly = (r / RE::X) % RE::Y - T::HE * T::HY;
    const int lz = r / (RE::X * RE::Y) - T::HE;
    const int jc = (lx + T::HJ) + (ly + T::HJ * T::HY) * sJy + (lz + T::HJ) * sJz;
    const int b = (lx + T::HB) + (ly + T::HB * T::HY) * sBy + (lz + T::HB) * sBz;
    const int gE = gidx(lx, ly, lz);
    const float4 mi = a.mom[gE];
    const float inv = 1.f / nf[jc];
    float bx = Bx[b], by = By[b], bz = Bz[b];
    if (a.B0) {  // the total field B0 + B1 in the cross products (and for the push)
      const float4 b0 = __ldg(a.B0 + gE);
      bx += b0.x;
      by += b0.y;
      bz += b0.z;
    }
    const float jx = Jx[jc], jy = Jy[jc], jz = Jz[jc];
    const float ux = jx - mi.y, uy = jy - mi.z, uz = jz - mi.w;
    const float qx = keep(x0 + lx, g.nx, g.open[0]), qz = keep(z0 + lz, g.nz, g.open[2]);
    const float qy = DIM == 2 ? 1.f : keep(y0 + ly, g.ny, g.open[1]);
    const float gpx = qx * (pe[jc + 1] - pe[jc - 1]) * k.idx2;
    const float gpy = DIM == 2 ? 0.f : qy * (pe[jc + sJy] - pe[jc - sJy]) * k.idy2;
    const float gpz = qz * (pe[jc + sJz] - pe[jc - sJz]) * k.idz2;
    float lx_ = qx * (Jx[jc + 1] + Jx[jc - 1] - 2.f * jx) * k.ilx +
                qz * (Jx[jc + sJz] + Jx[jc - sJz] - 2.f * jx) * k.ilz;
    float ly_ = qx * (Jy[jc + 1] + Jy[jc - 1] - 2.f * jy) * k.ilx +
                qz * (Jy[jc + sJz] + Jy[jc - sJz] - 2.f * jy) * k.ilz;
    float lz_ = qx * (Jz[jc + 1] + Jz[jc - 1] - 2.f * jz) * k.ilx +
                qz * (Jz[jc + sJz] + Jz[jc - sJz] - 2.f * jz) * k.ilz;
    if (DIM == 3) {
      lx_ += qy * (Jx[jc + sJy] + Jx[jc - sJy] - 2.f * jx) * k.ily;
      ly_ += qy * (Jy[jc + sJy] + Jy[jc - sJy] - 2.f * jy) * k.ily;
      lz_ += qy * (Jz[jc + sJy] + Jz[jc - sJy] - 2.f * jz) * k.ily;
    }
    float ex = ((uy * bz - uz * by) - gpx) * inv + k.eta * jx - k.eta_h * lx_;
    float ey = ((uz * bx - ux * bz) - gpy) * inv + k.eta * jy - k.eta_h * ly_;
    float ez = ((ux * by - uy * bx) - gpz) * inv + k.eta * jz - k.eta_h * lz_;
    if (k.model == 1) {  // electrostatic Ohm's law (Sec. 4): E = -grad p_e / n_f
      ex = -gpx * inv;
      ey = -gpy * inv;
      ez = -gpz * inv;
    } else if (k.model == 2) {  // resistive background (App. A): E = eta (J - J_k)
      ex = k.eta * (jx - mi.y);
      ey = k.eta * (jy - mi.z);
      ez = k.eta * (jz - mi.w);
    }
    if (FINAL) {
      // interior cell of the tile: write E, B into the padded gather array
      // at the cell and at each of its ghost images (with OPEN also the
      // ghost cells beyond the faces this tile touches)
      const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
      auto owns = [&](int gc, int org, int ext, int n, int open) {
        if (gc >= org && gc < org + ext && gc < n) return true;
        return OPEN && open && ((gc == -1 && org == 0) || (gc == n && org + ext >= n));
      };
      const bool mine = OPEN ? owns(gx, x0, T::OX, g.nx, g.open[0]) &&
                                   (DIM == 2 || owns(gy, y0, T::OY, g.ny, g.open[1])) &&
                                   owns(gz, z0, T::OZ, g.nz, g.open[2])
                             : (gx < g.nx && (DIM == 2 || gy < g.ny) && gz < g.nz);
      if (mine) {
        const float4 e0 = make_float4(ex, ey, ez, bx);
        const float4 e1 = make_float4(by, bz, 0.f, 0.f);
        if (OPEN) {
          int xs[5], ys[5], zs[5];
          const int nxs = (g.open[0] || gx < 0 || gx >= g.nx) ? (xs[0] = gx + kGhost, 1)
                                                               : axis_images(gx, g.nx, xs);
          int nys = 1;
          ys[0] = 0;
          if (DIM == 3)
            nys = (g.open[1] || gy < 0 || gy >= g.ny) ? (ys[0] = gy + kGhost, 1)
                                                      : axis_images(gy, g.ny, ys);
          const int nzs = (g.open[2] || gz < 0 || gz >= g.nz) ? (zs[0] = gz + kGhost, 1)
                                                               : axis_images(gz, g.nz, zs);
          for (int a3 = 0; a3 < nzs; ++a3)
            for (int a2 = 0; a2 < nys; ++a2)
              for (int a1 = 0; a1 < nxs; ++a1) {
                const int p = xs[a1] + (DIM == 2 ? 0 : ys[a2] * g.sy) + zs[a3] * g.sz;
                a.EB[2 * p] = e0;
                a.EB[2 * p + 1] = e1;
              }
          continue;
        }
        if (single_image(g, gx, gy, gz)) {
          const int p = voxel_of(g, gx, gy, gz);
          a.EB[2 * p] = e0;
          a.EB[2 * p + 1] = e1;
          continue;
        }
        int xs[5], ys[5], zs[5];
        const int nxs = axis_images(gx, g.nx, xs);
        const int nys = DIM == 2 ? 1 : axis_images(gy, g.ny, ys);
        if (DIM == 2) ys[0] = 0;
        const int nzs = axis_images(gz, g.nz, zs);
        for (int a3 = 0; a3 < nzs; ++a3)
          for (int a2 = 0; a2 < nys; ++a2)
            for (int a1 = 0; a1 < nxs; ++a1) {
              const int p = xs[a1] + (DIM == 2 ? 0 : ys[a2] * g.sy) + zs[a3] * g.sz;
              a.EB[2 * p] = e0;
              a.EB[2 * p + 1] = e1;
            }
      }
    } else {
      Ex[r] = ex;
      Ey[r] = ey;
      Ez[r] = ez;
      if (PEQ) {
        // electron flow u_e = -(J - J_i) / n_f, p_e u_e and T_e = p_e / n_f
        // (the electrostatic model has no magnetic current: u_e = J_i / n_f)
        const bool es = k.model == 1;
        const float jxm = es ? 0.f : jx, jym = es ? 0.f : jy, jzm = es ? 0.f : jz;
        const float ux_e = -(jxm - mi.y) * inv, uy_e = -(jym - mi.z) * inv,
                    uz_e = -(jzm - mi.w) * inv;
        const float p = pe[jc];
        Ux[r] = ux_e;
        Uy[r] = uy_e;
        Uz[r] = uz_e;
        Px[r] = p * ux_e;
        Py[r] = p * uy_e;
        Pz[r] = p * uz_e;
        Tel[r] = p * inv;
      }
    }
  }
  if (FINAL) return;
  __syncthreads();

  // B_out = B_base - coef * curl E on the tile (Eq. 5)
  constexpr int sEy = RE::X, sEz = RE::X * RE::Y;
  for (int r = threadIdx.x; r < T::OX * T::OY * T::OZ; r += blockDim.x) {
    const int lx = r % T::OX;
    const int ly = (r / T::OX) % T::OY;
    const int lz = r / (T::OX * T::OY);
    const int gx = x0 + lx, gy = y0 + ly, gz = z0 + lz;
    if (gx >= g.nx || (DIM == 3 && gy >= g.ny) || gz >= g.nz) continue;
    const int e = (lx + T::HE) + (ly + T::HE * T::HY) * sEy + (lz + T::HE) * sEz;
    const float dEz_dy = DIM == 2 ? 0.f : (Ez[e + sEy] - Ez[e - sEy]) * k.idy2;
    const float dEx_dy = DIM == 2 ? 0.f : (Ex[e + sEy] - Ex[e - sEy]) * k.idy2;
    const float dEy_dz = (Ey[e + sEz] - Ey[e - sEz]) * k.idz2;
    const float dEx_dz = (Ex[e + sEz] - Ex[e - sEz]) * k.idz2;
    const float dEz_dx = (Ez[e + 1] - Ez[e - 1]) * k.idx2;
    const float dEy_dx = (Ey[e + 1] - Ey[e - 1]) * k.idx2;
    const int c = gx + g.nx * ((DIM == 2 ? 0 : gy) + g.ny * gz);
    const float4 bb = a.Bbase[c];
    a.Bout[c] = make_float4(bb.x - a.coef * (dEz_dy - dEy_dz), bb.y - a.coef * (dEx_dz - dEz_dx),
                            bb.z - a.coef * (dEy_dx - dEx_dy), 0.f);
    if (PEQ) {
      // electron energy equation (Sec. 2.1, Eq. dpdt):
      //   dp_e/dt = -gamma div(p_e u_e) + (gamma-1) u_e . grad p_e
      //             + (gamma-1) kappa lap T_e
      constexpr int sJy_ = RJ::X, sJz_ = RJ::X * RJ::Y;
      const int jc = (lx + T::HJ) + (ly + T::HJ * T::HY) * sJy_ + (lz + T::HJ) * sJz_;
      float divpu = (Px[e + 1] - Px[e - 1]) * k.idx2 + (Pz[e + sEz] - Pz[e - sEz]) * k.idz2;
      float ugp = Ux[e] * (pe[jc + 1] - pe[jc - 1]) * k.idx2 +
                  Uz[e] * (pe[jc + sJz_] - pe[jc - sJz_]) * k.idz2;
      float lapT = (Tel[e + 1] + Tel[e - 1] - 2.f * Tel[e]) * k.ilx +
                   (Tel[e + sEz] + Tel[e - sEz] - 2.f * Tel[e]) * k.ilz;
      if (DIM == 3) {
        divpu += (Py[e + sEy] - Py[e - sEy]) * k.idy2;
        ugp += Uy[e] * (pe[jc + sJy_] - pe[jc - sJy_]) * k.idy2;
        lapT += (Tel[e + sEy] + Tel[e - sEy] - 2.f * Tel[e]) * k.ily;
      }
      const float gm1 = k.gamma_e - 1.f;
      const float dpdt = -k.gamma_e * divpu + gm1 * ugp + gm1 * k.kappa * lapT;
      a.pout[c] = a.pbase[c] + a.pcoef * dpdt;
    }
  }
}

// Electron pressure at start-up from the equation of state (Eq. 6) of the
// start-up moments, p_e = Te n_f^gamma_e.
__global__ void __launch_bounds__(256) pe_init_kernel(int ncell, FieldConsts k, const float4 *mom,
                                                      float *pe) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    const float f = fmaxf(mom[c].x, k.n_floor);
    pe[c] = k.isothermal ? k.Te * f : k.Te * powf(f, k.gamma_e);
  }
}

// ----------------------------------------------------------------------------
// One field stage in 3D (Eq. 5 with E from Eqs. 2-4, 6), streamed along z:
//   B_out = B_base - coef * curl E(B_in)
// A block owns an X x Y column of output cells over Z planes and walks up
// the column.  At step q it computes J = curl B on plane zj = z0 - 2 + q, E
// two planes behind and B_out two planes behind that, so every plane a step
// reads was written in an earlier step: one barrier per step suffices.  The
// planes of B and of the ion moments are fetched one step ahead with
// asynchronous copies into ring buffers, so no global load waits inside a
// step; only B_base is read from global memory, issued before the barrier.
// Every plane of B is loaded once per column and the halos are paid only in
// x and y.
//
// All planes share one layout: rows of P = X + 6 cells (the B halo of 3)
// and Y + 6 rows.  J (and n) is computed on rows 1..Y+4, E on rows 2..Y+3,
// over whole rows, so that the lanes of a warp touch consecutive words of
// shared memory; the values in the outer columns of those rows are never
// used.
// ----------------------------------------------------------------------------
#ifndef HV_ST3D_Z
#define HV_ST3D_Z 16
#endif
#ifndef HV_ST3D_THREADS
#define HV_ST3D_THREADS 384
#endif
namespace st3d {
constexpr int X = 32, Y = 8, Z = HV_ST3D_Z;  // output cells per block
constexpr int P = X + 6, R = Y + 6, NP = P * R;  // plane layout (B halo 3)
constexpr int J0 = P, NJ = P * (Y + 4);          // J, n: rows 1 .. Y+4
constexpr int E0 = 2 * P, NE = P * (Y + 2);      // E, moments: rows 2 .. Y+3
constexpr int kThreads = HV_ST3D_THREADS;
// ring depths: B planes zj-2..zj+2 (E reads zj-2, J zj-1..zj+1, the copy
// fills zj+2); J, p_e and E each hold three planes being read and one being
// written; n one plane read (by the J phase, for p_e) and one in flight; the
// moment float4 at E cells one read and one in flight
constexpr int kRB = 5, kRJ = 4, kRP = 4, kRN = 2, kRM = 2, kRE = 4;
constexpr int kB = 0;                    // [kRB][3][NP]
constexpr int kJ = kB + kRB * 3 * NP;    // [kRJ][3][NP]
constexpr int kP = kJ + kRJ * 3 * NP;    // [kRP][NP]   electron pressure p_e
constexpr int kN = kP + kRP * NP;        // [kRN][NP]   ion density n
constexpr int kM = kN + kRN * NP;        // [kRM][NP]   {n, Jix, Jiy, Jiz} as float4
constexpr int kE = kM + kRM * 4 * NP;    // [kRE][3][NP]
constexpr int kFloats = kE + kRE * 3 * NP;
static_assert(kM % 4 == 0, "moment ring must be 16-byte aligned");
}  // namespace st3d

__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

__global__ void __launch_bounds__(st3d::kThreads, 2) stage3d_kernel(StageArgs a) {
  pdl_begin();
  using namespace st3d;
  // cells per thread in each plane region; a thread keeps the x-y part of
  // its cells' global offsets, so a plane adds only its z offset
  constexpr int LB = (NP + kThreads - 1) / kThreads;
  constexpr int LJ = (NJ + kThreads - 1) / kThreads;
  constexpr int LE = (NE + kThreads - 1) / kThreads;
  constexpr int LO = (X * Y + kThreads - 1) / kThreads;
  extern __shared__ __align__(16) float sm[];
  const Geom &g = a.g;
  const FieldConsts &k = a.k;
  const int ntx = (g.nx + X - 1) / X, nty = (g.ny + Y - 1) / Y;
  const int bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, bz = blockIdx.x / (ntx * nty);
  const int x0 = bx * X, y0 = by * Y, z0 = bz * Z;
  const int t = threadIdx.x;
  const int sxy = g.nx * g.ny;
  // x-y part of the global offset of plane cell c (column c % P, row c / P)
  auto xy = [&](int c) {
    return wrap_near(x0 + c % P - 3, g.nx, X + 3) + g.nx * wrap_near(y0 + c / P - 3, g.ny, Y + 3);
  };
  auto zoff = [&](int z) { return sxy * wrap_near(z, g.nz, Z + 6); };
  // ring slot of plane z (planes start at z0 - 3, so the index is >= 0)
  auto slot = [&](int z, int depth) { return (z - z0 + 8) % depth; };
  int xb[LB], xj[LJ], xe[LE], xo[LO];
#pragma unroll
  for (int u = 0; u < LB; ++u) {
    const int r = t + u * kThreads;
    xb[u] = r < NP ? xy(r) : 0;
  }
#pragma unroll
  for (int u = 0; u < LJ; ++u) {
    const int r = t + u * kThreads;
    xj[u] = r < NJ ? xy(J0 + r) : 0;
  }
#pragma unroll
  for (int u = 0; u < LE; ++u) {
    const int r = t + u * kThreads;
    xe[u] = r < NE ? xy(E0 + r) : 0;
  }
#pragma unroll
  for (int u = 0; u < LO; ++u) {
    const int r = t + u * kThreads;
    const int gx = x0 + r % X, gy = y0 + r / X;
    xo[u] = (r < X * Y && gx < g.nx && gy < g.ny) ? gx + g.nx * gy : -1;
  }
  auto copy_B = [&](int z) {
    float *b = sm + kB + slot(z, kRB) * 3 * NP;
    const int zo_ = zoff(z);
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int r = t + u * kThreads;
      if (r >= NP) continue;
      const float *src = reinterpret_cast<const float *>(a.Bin + (xb[u] + zo_));
      cp_async4(b + r, src);
      cp_async4(b + NP + r, src + 1);
      cp_async4(b + 2 * NP + r, src + 2);
    }
  };
  auto copy_n = [&](int z) {
    float *nn = sm + kN + slot(z, kRN) * NP + J0;
    const int zo_ = zoff(z);
#pragma unroll
    for (int u = 0; u < LJ; ++u) {
      const int r = t + u * kThreads;
      if (r < NJ) cp_async4(nn + r, reinterpret_cast<const float *>(a.mom + (xj[u] + zo_)));
    }
  };
  auto copy_m = [&](int z) {
    float4 *m = reinterpret_cast<float4 *>(sm + kM) + slot(z, kRM) * NP + E0;
    const int zo_ = zoff(z);
#pragma unroll
    for (int u = 0; u < LE; ++u) {
      const int r = t + u * kThreads;
      if (r < NE) cp_async16(m + r, a.mom + (xe[u] + zo_));
    }
  };
  // electron pressure p_e(n) with the density floor (Eq. 4)
  auto pe = [&](float n) {
    const float f = fmaxf(n, k.n_floor);
    return k.isothermal ? k.Te * f : k.Te * powf(f, k.gamma_e);
  };

  copy_B(z0 - 3);
  copy_B(z0 - 2);
  copy_B(z0 - 1);
  copy_n(z0 - 2);
  cp_async_commit();
  for (int q = 0; q < Z + 6; ++q) {
    const int zj = z0 - 2 + q, ze = zj - 2, zo = ze - 2;
    const bool out_on = q >= 6 && zo < g.nz;
    // B_base of the output plane: only this thread reads or writes these
    // cells, so the load may precede the barrier even when B_out == B_base
    float4 bb[LO];
#pragma unroll
    for (int u = 0; u < LO; ++u)
      bb[u] = (out_on && xo[u] >= 0) ? a.Bbase[xo[u] + sxy * zo] : make_float4(0.f, 0.f, 0.f, 0.f);
    cp_async_wait_all();
    __syncthreads();
    // one step ahead: B for the next J plane, n and the moments for the
    // next E plane
    if (q <= Z + 2) copy_B(zj + 2);
    if (q <= Z + 2) copy_n(zj + 1);
    if (q >= 2 && q <= Z + 3) copy_m(ze + 1);
    cp_async_commit();

    if (q <= Z + 3) {  // J = curl B and p_e on plane zj
      const float *bm = sm + kB + slot(zj - 1, kRB) * 3 * NP;
      const float *b0 = sm + kB + slot(zj, kRB) * 3 * NP;
      const float *bp = sm + kB + slot(zj + 1, kRB) * 3 * NP;
      const float *nn = sm + kN + slot(zj, kRN) * NP;
      float *j = sm + kJ + slot(zj, kRJ) * 3 * NP;
      float *pp = sm + kP + slot(zj, kRP) * NP;
#pragma unroll
      for (int u = 0; u < LJ; ++u) {
        const int r = t + u * kThreads;
        if (r >= NJ) continue;
        const int c = J0 + r;
        const float dBz_dy = (b0[2 * NP + c + P] - b0[2 * NP + c - P]) * k.idy2;
        const float dBx_dy = (b0[c + P] - b0[c - P]) * k.idy2;
        const float dBy_dz = (bp[NP + c] - bm[NP + c]) * k.idz2;
        const float dBx_dz = (bp[c] - bm[c]) * k.idz2;
        const float dBz_dx = (b0[2 * NP + c + 1] - b0[2 * NP + c - 1]) * k.idx2;
        const float dBy_dx = (b0[NP + c + 1] - b0[NP + c - 1]) * k.idx2;
        j[c] = dBz_dy - dBy_dz;
        j[NP + c] = dBx_dz - dBz_dx;
        j[2 * NP + c] = dBy_dx - dBx_dy;
        pp[c] = pe(nn[c]);
      }
    }
    if (q >= 3 && q <= Z + 4) {  // E from Ohm's law on plane ze
      const float *jm = sm + kJ + slot(ze - 1, kRJ) * 3 * NP;
      const float *j0 = sm + kJ + slot(ze, kRJ) * 3 * NP;
      const float *jp = sm + kJ + slot(ze + 1, kRJ) * 3 * NP;
      const float *pm = sm + kP + slot(ze - 1, kRP) * NP;
      const float *p0 = sm + kP + slot(ze, kRP) * NP;
      const float *pq = sm + kP + slot(ze + 1, kRP) * NP;
      const float4 *m0 = reinterpret_cast<const float4 *>(sm + kM) + slot(ze, kRM) * NP;
      const float *b0 = sm + kB + slot(ze, kRB) * 3 * NP;
      float *e = sm + kE + slot(ze, kRE) * 3 * NP;
#pragma unroll
      for (int u = 0; u < LE; ++u) {
        const int r = t + u * kThreads;
        if (r >= NE) continue;
        const int c = E0 + r;
        const float4 mi = m0[c];
        const float inv = __frcp_rn(fmaxf(mi.x, k.n_floor));
        float bxv = b0[c], byv = b0[NP + c], bzv = b0[2 * NP + c];
        if (a.B0) {  // total field B0 + B1 in the cross products
          const float4 ext = __ldg(a.B0 + xe[u] + zoff(ze));
          bxv += ext.x;
          byv += ext.y;
          bzv += ext.z;
        }
        const float jx = j0[c], jy = j0[NP + c], jz = j0[2 * NP + c];
        const float ux = jx - mi.y, uy = jy - mi.z, uz = jz - mi.w;
        const float gpx = (p0[c + 1] - p0[c - 1]) * k.idx2;
        const float gpy = (p0[c + P] - p0[c - P]) * k.idy2;
        const float gpz = (pq[c] - pm[c]) * k.idz2;
        float l[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const float c0 = j0[m * NP + c];
          l[m] = (j0[m * NP + c + 1] + j0[m * NP + c - 1] - 2.f * c0) * k.ilx +
                 (j0[m * NP + c + P] + j0[m * NP + c - P] - 2.f * c0) * k.ily +
                 (jp[m * NP + c] + jm[m * NP + c] - 2.f * c0) * k.ilz;
        }
        e[c] = ((uy * bzv - uz * byv) - gpx) * inv + k.eta * jx - k.eta_h * l[0];
        e[NP + c] = ((uz * bxv - ux * bzv) - gpy) * inv + k.eta * jy - k.eta_h * l[1];
        e[2 * NP + c] = ((ux * byv - uy * bxv) - gpz) * inv + k.eta * jz - k.eta_h * l[2];
      }
    }
    if (out_on) {  // B_out = B_base - coef * curl E on plane zo
      const float *em = sm + kE + slot(zo - 1, kRE) * 3 * NP;
      const float *e0 = sm + kE + slot(zo, kRE) * 3 * NP;
      const float *ep = sm + kE + slot(zo + 1, kRE) * 3 * NP;
      const int zo_ = sxy * zo;
#pragma unroll
      for (int u = 0; u < LO; ++u) {
        const int r = t + u * kThreads;
        if (xo[u] < 0) continue;
        const int c = (r % X + 3) + (r / X + 3) * P;
        const float dEz_dy = (e0[2 * NP + c + P] - e0[2 * NP + c - P]) * k.idy2;
        const float dEx_dy = (e0[c + P] - e0[c - P]) * k.idy2;
        const float dEy_dz = (ep[NP + c] - em[NP + c]) * k.idz2;
        const float dEx_dz = (ep[c] - em[c]) * k.idz2;
        const float dEz_dx = (e0[2 * NP + c + 1] - e0[2 * NP + c - 1]) * k.idx2;
        const float dEy_dx = (e0[NP + c + 1] - e0[NP + c - 1]) * k.idx2;
        a.Bout[xo[u] + zo_] =
            make_float4(bb[u].x - a.coef * (dEz_dy - dEy_dz), bb[u].y - a.coef * (dEx_dz - dEz_dx),
                        bb[u].z - a.coef * (dEy_dx - dEx_dy), 0.f);
      }
    }
  }
}

// ----------------------------------------------------------------------------
// One whole explicit-midpoint substep in the x-z layout, fused:
//   B* = B - (h/2) curl E(B),  B_out = B - h curl E(B*)
// A 32x16 tile of outputs needs B on a halo of 6 cells: each Ohm evaluation
// reaches 2 cells (J = curl B, then lap J) and each curl of E one more.
// Every input is loaded once into shared memory; both stages then run from
// there.
//
// Each thread takes two x-adjacent cells at a time: the pair's own and its
// z-neighbours' operands are one 8-byte shared load for both cells, and only
// the two outer x-neighbours are single loads.  For that every array starts
// at an even x and has an even width; a region whose halo is odd grows by a
// column on each side.  Those extra columns read one cell past the end of
// their row (still inside the array) and hold values that no valid cell of
// the next stage reads.
// ----------------------------------------------------------------------------
namespace sub2d {
constexpr int SX = 32, SZ = 16, SH = 6;
// tile-local array over x in [OX, OX + WW), z in [OZ, OZ + HH), row-major
template <int OX, int WW, int OZ, int HH>
struct Reg {
  static_assert(OX % 2 == 0 && WW % 2 == 0, "cell pairs start at an even x");
  static constexpr int ox = OX, w = WW, oz = OZ, h = HH, n = WW * HH, pairs = WW / 2 * HH;
  __device__ static __forceinline__ int at(int x, int z) { return (x - OX) + (z - OZ) * WW; }
};
using RB = Reg<-6, SX + 12, -6, SZ + 12>;   // B
using RM = Reg<-6, SX + 12, -5, SZ + 10>;   // p_e, 1/n_f, J_i
using RJ1 = Reg<-6, SX + 12, -5, SZ + 10>;  // J = curl B, valid on x in [-5, SX + 5)
using RE1 = Reg<-4, SX + 8, -4, SZ + 8>;    // E(B)
using RS = Reg<-4, SX + 8, -3, SZ + 6>;     // B*, valid on x in [-3, SX + 3)
using RJ2 = Reg<-2, SX + 4, -2, SZ + 4>;    // J = curl B*
using RE2 = Reg<-2, SX + 4, -1, SZ + 2>;    // E(B*), valid on x in [-1, SX + 1)
using R0 = Reg<0, SX, 0, SZ>;               // B_out
constexpr int kB = 0;                       // B (3 planes)
constexpr int kM = kB + 3 * RB::n;          // p_e, 1/n_f, Jix, Jiy, Jiz
constexpr int kJ = kM + 5 * RM::n;          // J (stage 1, then stage 2)
constexpr int kE = kJ + 3 * RJ1::n;         // E (stage 1, then stage 2)
constexpr int kS = kE + 3 * RE1::n;         // B*
constexpr int kFloats = kS + 3 * RS::n;
static_assert(RJ2::n <= RJ1::n && RE2::n <= RE1::n, "stage 2 reuses the stage-1 arrays");
static_assert(RB::n % 2 == 0 && RM::n % 2 == 0 && RJ1::n % 2 == 0 && RE1::n % 2 == 0 &&
                  RS::n % 2 == 0 && RJ2::n % 2 == 0 && RE2::n % 2 == 0,
              "every plane starts 8-byte aligned");
__device__ __forceinline__ float2 ld2(const float *p) {
  return *reinterpret_cast<const float2 *>(p);
}
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
struct Pair3 {
  float2 x, y, z;
};
// curl V at cells (x, z) and (x + 1, z) from V on region R (y derivatives
// vanish in the x-z layout): J = curl B and the curl of E in Faraday's law
template <class R>
__device__ __forceinline__ Pair3 curl_pair(const FieldConsts &k, const float *V, int x, int z) {
  const float *Vx = V, *Vy = V + R::n, *Vz = V + 2 * R::n;
  const int b = R::at(x, z), w = R::w;
  const float2 yu = ld2(Vy + b + w), yd = ld2(Vy + b - w), yc = ld2(Vy + b);
  const float2 xu = ld2(Vx + b + w), xd = ld2(Vx + b - w), zc = ld2(Vz + b);
  const float yl = Vy[b - 1], yr = Vy[b + 2], zl = Vz[b - 1], zr = Vz[b + 2];
  Pair3 c;
  c.x = make_float2(-(yu.x - yd.x) * k.idz2, -(yu.y - yd.y) * k.idz2);
  c.y = make_float2((xu.x - xd.x) * k.idz2 - (zc.y - zl) * k.idx2,
                    (xu.y - xd.y) * k.idz2 - (zr - zc.x) * k.idx2);
  c.z = make_float2((yc.y - yl) * k.idx2, (yr - yc.x) * k.idx2);
  return c;
}
}  // namespace sub2d

struct SubArgs {
  Geom g;
  FieldConsts k;
  const float4 *B;
  float4 *Bout;
  const float4 *mom;
  const float4 *B0;  // external field (interior) or null
  float h;
};

// E from Ohm's law at one cell from its operands: the pressure gradient, J
// and lap J, the total B, the ion current J_i and 1/n_f.
__device__ __forceinline__ void ohm_cell(const FieldConsts &k, float gpx, float gpz, float jx,
                                         float jy, float jz, float lx, float ly, float lz,
                                         float bx, float by, float bz, float mx, float my,
                                         float mz, float inv, float &ex, float &ey, float &ez) {
  const float ux = jx - mx, uy = jy - my, uz = jz - mz;
  ex = ((uy * bz - uz * by) - gpx) * inv + k.eta * jx - k.eta_h * lx;
  ey = (uz * bx - ux * bz) * inv + k.eta * jy - k.eta_h * ly;
  ez = ((ux * by - uy * bx) - gpz) * inv + k.eta * jz - k.eta_h * lz;
}

// E from Ohm's law at cells (x, z), (x + 1, z), with B on region RBs, J on
// RJs, and p_e, 1/n_f, J_i per cell (computed once per cell at load).  With
// an external field (B = B0 + B1 split, Sec. 2.3) Bp holds B1 and b0, b1 are
// B0 at the two cells: J = curl B1, the cross products take the total field.
template <class RBs, class RJs>
__device__ __forceinline__ void ohm_pair(const float *sm, const FieldConsts &k, int x, int z,
                                         const float *Bp, const float *Jp, float4 b0, float4 b1,
                                         sub2d::Pair3 &e) {
  using namespace sub2d;
  const float *pe = sm + kM, *invn = pe + RM::n, *mjx = invn + RM::n, *mjy = mjx + RM::n,
              *mjz = mjy + RM::n;
  const int im = RM::at(x, z);
  const float2 pc = ld2(pe + im), pu = ld2(pe + im + RM::w), pd = ld2(pe + im - RM::w);
  const float pl = pe[im - 1], pr = pe[im + 2];
  const float2 nv = ld2(invn + im), m_x = ld2(mjx + im), m_y = ld2(mjy + im),
               m_z = ld2(mjz + im);
  const int ij = RJs::at(x, z), wj = RJs::w;
  float2 jc[3], lp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float *J = Jp + c * RJs::n;
    const float2 cc = ld2(J + ij), uu = ld2(J + ij + wj), dd = ld2(J + ij - wj);
    const float l = J[ij - 1], r = J[ij + 2];
    jc[c] = cc;
    lp[c] = make_float2((cc.y + l - 2.f * cc.x) * k.ilx + (uu.x + dd.x - 2.f * cc.x) * k.ilz,
                        (r + cc.x - 2.f * cc.y) * k.ilx + (uu.y + dd.y - 2.f * cc.y) * k.ilz);
  }
  const int ib = RBs::at(x, z);
  const float2 bx = ld2(Bp + ib), by = ld2(Bp + RBs::n + ib), bz = ld2(Bp + 2 * RBs::n + ib);
  ohm_cell(k, (pc.y - pl) * k.idx2, (pu.x - pd.x) * k.idz2, jc[0].x, jc[1].x, jc[2].x, lp[0].x,
           lp[1].x, lp[2].x, bx.x + b0.x, by.x + b0.y, bz.x + b0.z, m_x.x, m_y.x, m_z.x, nv.x,
           e.x.x, e.y.x, e.z.x);
  ohm_cell(k, (pr - pc.x) * k.idx2, (pu.y - pd.y) * k.idz2, jc[0].y, jc[1].y, jc[2].y, lp[0].y,
           lp[1].y, lp[2].y, bx.y + b1.x, by.y + b1.y, bz.y + b1.z, m_x.y, m_y.y, m_z.y, nv.y,
           e.x.y, e.y.y, e.z.y);
}

// threads per block of the fused subcycle kernel
#ifndef HV_SUB_THREADS
#define HV_SUB_THREADS 384
#endif
constexpr int kSubThreads = HV_SUB_THREADS;

// f(x, z) for every cell pair (x, z), (x + 1, z) of region R, pairs spread
// over the block's threads in row-major order
template <class R, class F>
__device__ __forceinline__ void for_pairs(F f) {
  for (int t = (int)threadIdx.x; t < R::pairs; t += kSubThreads)
    f(R::ox + 2 * (t % (R::w / 2)), R::oz + t / (R::w / 2));
}

__global__ void __launch_bounds__(kSubThreads) substep2d_kernel(SubArgs a) {
  pdl_begin();
  using namespace sub2d;
  extern __shared__ __align__(16) float sm[];
  const Geom &g = a.g;
  const FieldConsts &k = a.k;
  const int ntx = (g.nx + SX - 1) / SX;
  const int x0 = (blockIdx.x % ntx) * SX, z0 = (blockIdx.x / ntx) * SZ;
  float *Bp = sm + kB, *Mp = sm + kM, *Jp = sm + kJ, *Ep = sm + kE, *Sp = sm + kS;
  auto gidx = [&](int x, int z) {
    const int ii = wrap_near(x0 + x, g.nx, SX + SH);
    const int kk = wrap_near(z0 + z, g.nz, SZ + SH);
    return ii + g.nx * kk;
  };
  // load B on RB and the moments on RM, two cells per pair: every thread
  // issues all its loads before it stores any, so the L2 latencies overlap
  {
    constexpr int LB = (RB::pairs + kSubThreads - 1) / kSubThreads;
    constexpr int LM = (RM::pairs + kSubThreads - 1) / kSubThreads;
    float4 bv[2 * LB], mv[2 * LM];
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int t = (int)threadIdx.x + u * kSubThreads;
      if (t < RB::pairs) {
        const int x = RB::ox + 2 * (t % (RB::w / 2)), z = RB::oz + t / (RB::w / 2);
        bv[2 * u] = a.B[gidx(x, z)];
        bv[2 * u + 1] = a.B[gidx(x + 1, z)];
      }
    }
#pragma unroll
    for (int u = 0; u < LM; ++u) {
      const int t = (int)threadIdx.x + u * kSubThreads;
      if (t < RM::pairs) {
        const int x = RM::ox + 2 * (t % (RM::w / 2)), z = RM::oz + t / (RM::w / 2);
        mv[2 * u] = a.mom[gidx(x, z)];
        mv[2 * u + 1] = a.mom[gidx(x + 1, z)];
      }
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int t = (int)threadIdx.x + u * kSubThreads;
      if (t < RB::pairs) {
        const int i = 2 * t;  // the pair's index in row-major order
        const float4 c0 = bv[2 * u], c1 = bv[2 * u + 1];
        st2(Bp + i, make_float2(c0.x, c1.x));
        st2(Bp + RB::n + i, make_float2(c0.y, c1.y));
        st2(Bp + 2 * RB::n + i, make_float2(c0.z, c1.z));
      }
    }
#pragma unroll
    for (int u = 0; u < LM; ++u) {
      const int t = (int)threadIdx.x + u * kSubThreads;
      if (t < RM::pairs) {
        const int i = 2 * t;
        const float4 c0 = mv[2 * u], c1 = mv[2 * u + 1];
        // p_e and 1/n_f once per cell (the floor enters both, Sec. 2.1)
        const float f0 = fmaxf(c0.x, k.n_floor), f1 = fmaxf(c1.x, k.n_floor);
        st2(Mp + i, k.isothermal ? make_float2(k.Te * f0, k.Te * f1)
                                 : make_float2(k.Te * powf(f0, k.gamma_e),
                                               k.Te * powf(f1, k.gamma_e)));
        st2(Mp + RM::n + i, make_float2(__frcp_rn(f0), __frcp_rn(f1)));
        st2(Mp + 2 * RM::n + i, make_float2(c0.y, c1.y));
        st2(Mp + 3 * RM::n + i, make_float2(c0.z, c1.z));
        st2(Mp + 4 * RM::n + i, make_float2(c0.w, c1.w));
      }
    }
  }
  __syncthreads();
  // stage 1: J(B), E(B), B* = B - (h/2) curl E
  for_pairs<RJ1>([&](int x, int z) {
    const Pair3 c = curl_pair<RB>(k, Bp, x, z);
    const int j = RJ1::at(x, z);
    st2(Jp + j, c.x);
    st2(Jp + RJ1::n + j, c.y);
    st2(Jp + 2 * RJ1::n + j, c.z);
  });
  __syncthreads();
  for_pairs<RE1>([&](int x, int z) {
    float4 b0 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = b0;
    if (a.B0) {
      b0 = __ldg(a.B0 + gidx(x, z));
      b1 = __ldg(a.B0 + gidx(x + 1, z));
    }
    Pair3 e;
    ohm_pair<RB, RJ1>(sm, k, x, z, Bp, Jp, b0, b1, e);
    const int i = RE1::at(x, z);
    st2(Ep + i, e.x);
    st2(Ep + RE1::n + i, e.y);
    st2(Ep + 2 * RE1::n + i, e.z);
  });
  __syncthreads();
  const float c1 = 0.5f * a.h;
  for_pairs<RS>([&](int x, int z) {
    const Pair3 c = curl_pair<RE1>(k, Ep, x, z);
    const int b = RB::at(x, z), s = RS::at(x, z);
    const float2 bx = ld2(Bp + b), by = ld2(Bp + RB::n + b), bz = ld2(Bp + 2 * RB::n + b);
    st2(Sp + s, make_float2(bx.x - c1 * c.x.x, bx.y - c1 * c.x.y));
    st2(Sp + RS::n + s, make_float2(by.x - c1 * c.y.x, by.y - c1 * c.y.y));
    st2(Sp + 2 * RS::n + s, make_float2(bz.x - c1 * c.z.x, bz.y - c1 * c.z.y));
  });
  __syncthreads();
  // stage 2: J(B*), E(B*), B_out = B - h curl E
  for_pairs<RJ2>([&](int x, int z) {
    const Pair3 c = curl_pair<RS>(k, Sp, x, z);
    const int j = RJ2::at(x, z);
    st2(Jp + j, c.x);
    st2(Jp + RJ2::n + j, c.y);
    st2(Jp + 2 * RJ2::n + j, c.z);
  });
  __syncthreads();
  for_pairs<RE2>([&](int x, int z) {
    float4 b0 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = b0;
    if (a.B0) {
      b0 = __ldg(a.B0 + gidx(x, z));
      b1 = __ldg(a.B0 + gidx(x + 1, z));
    }
    Pair3 e;
    ohm_pair<RS, RJ2>(sm, k, x, z, Sp, Jp, b0, b1, e);
    const int i = RE2::at(x, z);
    st2(Ep + i, e.x);
    st2(Ep + RE2::n + i, e.y);
    st2(Ep + 2 * RE2::n + i, e.z);
  });
  __syncthreads();
  for_pairs<R0>([&](int x, int z) {
    const int gx = x0 + x, gz = z0 + z;
    if (gz >= g.nz || gx >= g.nx) return;
    const Pair3 c = curl_pair<RE2>(k, Ep, x, z);
    const int b = RB::at(x, z);
    const float2 bx = ld2(Bp + b), by = ld2(Bp + RB::n + b), bz = ld2(Bp + 2 * RB::n + b);
    float4 *out = a.Bout + gx + g.nx * gz;
    out[0] = make_float4(bx.x - a.h * c.x.x, by.x - a.h * c.y.x, bz.x - a.h * c.z.x, 0.f);
    if (gx + 1 < g.nx)
      out[1] = make_float4(bx.y - a.h * c.x.y, by.y - a.h * c.y.y, bz.y - a.h * c.z.y, 0.f);
  });
}

FieldConsts field_consts(const hv_ctx *c) {
  FieldConsts k;
  const hv_params &p = c->p;
  k.idx2 = p.nx > 1 ? (float)(1.0 / (2.0 * p.dx)) : 0.f;
  k.idy2 = p.ny > 1 ? (float)(1.0 / (2.0 * p.dy)) : 0.f;
  k.idz2 = p.nz > 1 ? (float)(1.0 / (2.0 * p.dz)) : 0.f;
  k.ilx = p.nx > 1 ? (float)(1.0 / (p.dx * p.dx)) : 0.f;
  k.ily = p.ny > 1 ? (float)(1.0 / (p.dy * p.dy)) : 0.f;
  k.ilz = p.nz > 1 ? (float)(1.0 / (p.dz * p.dz)) : 0.f;
  k.Te = (float)p.Te;
  k.gamma_e = (float)p.gamma_e;
  k.eta = (float)p.eta;
  k.eta_h = (float)p.eta_h;
  k.n_floor = (float)p.n_floor;
  k.isothermal = p.gamma_e == 1.0;
  k.kappa = (float)p.kappa;
  k.model = p.ohm_model;
  return k;
}

template <int DIM, int FINAL, int PEQ = 0, int OPEN = 0>
cudaError_t launch_stage_t(const hv_ctx *c, const StageArgs &a) {
  using T = Tile<DIM, FINAL, PEQ, OPEN>;
  const size_t smem = T::smem_floats * sizeof(float);
  static std::atomic<uint64_t> attr_set{0};
  cudaError_t e = set_smem_once(stage_kernel<DIM, FINAL, PEQ, OPEN>, smem, attr_set);
  if (e != cudaSuccess) return e;
  const int ntx = (c->g.nx + T::OX - 1) / T::OX;
  const int nty = DIM == 2 ? 1 : (c->g.ny + T::OY - 1) / T::OY;
  const int ntz = (c->g.nz + T::OZ - 1) / T::OZ;
  return launch_pdl(stage_kernel<DIM, FINAL, PEQ, OPEN>, ntx * nty * ntz, 256, smem, c->stream,
                    a);
}

// ----------------------------------------------------------------------------
// diagnostics
// ----------------------------------------------------------------------------

// W_B of the total field (B0 + B1 with an external field), max |div| of the
// advanced field B (B1 with an external field), charge of the moments.
// Per cell in FP32, summed per thread and block in FP64 (the conservation
// sums): 1/2 |B|^2 of the total field, the charge density, and the largest
// |div B| of the advanced field B (B1 with an external field; max is exact
// in any precision, the divergence itself is FP32).  Block partials, not
// yet multiplied by the cell volume: {W_B, charge, max |div B|, 0}.
__global__ void __launch_bounds__(256) grid_diag_kernel(Geom g, FieldConsts k, const float4 *B,
                                                        const float4 *B0, const float4 *mom,
                                                        double *part) {
  double wb = 0.0, ch = 0.0;
  float md = 0.f;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += gridDim.x * blockDim.x) {
    int i, j, kk;
    decode(g, c, i, j, kk);
    float4 b = B[c];
    if (B0) {
      const float4 e = B0[c];
      b = make_float4(b.x + e.x, b.y + e.y, b.z + e.z, 0.f);
    }
    wb += (double)(0.5f * (b.x * b.x + b.y * b.y + b.z * b.z));
    ch += (double)mom[c].x;
    // neighbours: periodic images, or on an open axis the cell itself beyond
    // the face (the ghost copies its interior neighbour)
    auto nb = [](int c, int n, int open) {
      return open ? (c < 0 ? 0 : (c >= n ? n - 1 : c)) : wrapn(c, n);
    };
    const int xp = nb(i + 1, g.nx, g.open[0]) + g.nx * (j + g.ny * kk);
    const int xm = nb(i - 1, g.nx, g.open[0]) + g.nx * (j + g.ny * kk);
    const int yp = i + g.nx * (nb(j + 1, g.ny, g.open[1]) + g.ny * kk);
    const int ym = i + g.nx * (nb(j - 1, g.ny, g.open[1]) + g.ny * kk);
    const int zp = i + g.nx * (j + g.ny * nb(kk + 1, g.nz, g.open[2]));
    const int zm = i + g.nx * (j + g.ny * nb(kk - 1, g.nz, g.open[2]));
    const float dv = (B[xp].x - B[xm].x) * k.idx2 + (B[yp].y - B[ym].y) * k.idy2 +
                     (B[zp].z - B[zm].z) * k.idz2;
    md = fmaxf(md, fabsf(dv));
  }
  // the warp's lanes, then the block's warps, in a fixed order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    wb += __shfl_down_sync(0xffffffffu, wb, o);
    ch += __shfl_down_sync(0xffffffffu, ch, o);
    md = fmaxf(md, __shfl_down_sync(0xffffffffu, md, o));
  }
  __shared__ double s[3][8];
  if (lane == 0) {
    s[0][warp] = wb;
    s[1][warp] = ch;
    s[2][warp] = md;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double r = s[threadIdx.x][0];
    for (int w = 1; w < 8; ++w) r = threadIdx.x == 2 ? fmax(r, s[2][w]) : r + s[threadIdx.x][w];
    part[blockIdx.x * 4 + threadIdx.x] = r;
    if (threadIdx.x == 0) part[blockIdx.x * 4 + 3] = 0.0;
  }
}

// Fixed-order sums of the grid and particle partials, spread over
// kDiagBlocks blocks: each block sums a fixed slice of the partials and
// writes its result; the block that finishes last (a counter, no waiting)
// adds the block results in block order and rearms the counter.
// out: W_K, Px, Py, Pz, charge, W_B, max_divB
constexpr int kDiagThreads = 256;
__global__ void __launch_bounds__(kDiagThreads)
    diag_final_kernel(const double *gpart, int ngb, const double *ppart, int nppart,
                      double vc, double *blk, unsigned *count, double *out) {
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  const int nb = gridDim.x;
  const int g0 = (int)((int64_t)ngb * blockIdx.x / nb), g1 = (int)((int64_t)ngb * (blockIdx.x + 1) / nb);
  const int p0 = (int)((int64_t)nppart * blockIdx.x / nb),
            p1 = (int)((int64_t)nppart * (blockIdx.x + 1) / nb);
  for (int b = g0 + threadIdx.x; b < g1; b += blockDim.x) {
    v[5] += gpart[b * 4 + 0];
    v[4] += gpart[b * 4 + 1];
    v[6] = fmax(v[6], gpart[b * 4 + 2]);
  }
  const double4 *pp = reinterpret_cast<const double4 *>(ppart);
  for (int b = p0 + threadIdx.x; b < p1; b += blockDim.x) {
    const double4 q = pp[b];
    v[0] += q.x;
    v[1] += q.y;
    v[2] += q.z;
    v[3] += q.w;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int m = 0; m < 6; ++m) v[m] += __shfl_down_sync(0xffffffffu, v[m], o);
    v[6] = fmax(v[6], __shfl_down_sync(0xffffffffu, v[6], o));
  }
  __shared__ double s[7][kDiagThreads / 32];
  __shared__ bool last;
  if (lane == 0)
    for (int m = 0; m < 7; ++m) s[m][warp] = v[m];
  __syncthreads();
  if (threadIdx.x < 7) {
    double r = s[threadIdx.x][0];
    for (int w = 1; w < kDiagThreads / 32; ++w)
      r = threadIdx.x == 6 ? fmax(r, s[6][w]) : r + s[threadIdx.x][w];
    blk[blockIdx.x * 8 + threadIdx.x] = r;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(count, 1u) == (unsigned)(nb - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  // every block's results into shared memory with one load per thread,
  // then the sums in block order
  __shared__ double sb[kDiagBlocks * 8];
  const volatile double *vb = blk;
  for (int e = threadIdx.x; e < nb * 8; e += blockDim.x) sb[e] = vb[e];
  __syncthreads();
  if (threadIdx.x < 7) {
    double r = sb[threadIdx.x];
    for (int b = 1; b < nb; ++b)
      r = threadIdx.x == 6 ? fmax(r, sb[b * 8 + 6]) : r + sb[b * 8 + threadIdx.x];
    // the grid sums are per unit volume until here
    out[threadIdx.x] = (threadIdx.x == 4 || threadIdx.x == 5) ? r * vc : r;
  }
  if (threadIdx.x == 0) *count = 0u;
}

}  // namespace

int grid_reduce_blocks(int device) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return sms > 0 ? 8 * sms : 8;
}

static int elem_blocks(int n) {
  int b = (n + 255) / 256;
  return b < 1 ? 1 : (b > 4096 ? 4096 : b);
}

// `passes` binomial passes of the float4 grid in x, with y as scratch;
// *res receives whichever of the two holds the result.  The x-z layout
// runs up to smz::kMax passes per launch.
static cudaError_t smooth_grid(hv_ctx *c, float4 *x, float4 *y, int passes, float4 **res) {
  const Geom &g = c->g;
  const bool fused = g.dim2;
  static std::atomic<uint64_t> attr_set{0};
  if (fused) {
    cudaError_t e = set_smem_once(smooth2d_multi_kernel, smz::kBytes, attr_set);
    if (e != cudaSuccess) return e;
  }
  const int nb = elem_blocks(g.ncell);
  const int tiles = ((g.nx + smz::T - 1) / smz::T) * ((g.nz + smz::T - 1) / smz::T);
  for (int done = 0; done < passes;) {
    const int k = fused ? std::min(passes - done, smz::kMax) : 1;
    c->launches++;
    if (fused)
      smooth2d_multi_kernel<<<tiles, smz::kThreads, smz::kBytes, c->stream>>>(g, x, y, k);
    else
      smooth_kernel<<<nb, 256, 0, c->stream>>>(g, x, y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    std::swap(x, y);
    done += k;
  }
  *res = x;
  return cudaSuccess;
}

cudaError_t launch_moments(hv_ctx *c, int init) {
  MomArgs a;
  a.g = c->g;
  a.acc = c->acc;
  a.rec = c->accm[c->accpar];
  a.prev_in = c->mprev;
  a.prev_out = c->mprev;
  a.ext_out = c->mext;
  a.raw_out = c->mtmp;
  a.init = init;
  const int passes = c->filter_on ? 0 : c->p.smooth_passes;
  a.fuse = passes == 0 && !c->filter_on;
  const int nb = elem_blocks(c->g.ncell);
  c->launches++;
  if (uses_records(c)) {
    cudaError_t el = launch_pdl(fold_records_kernel, nb, 256, 0, c->stream, a);
    if (el != cudaSuccess) return el;
    c->accpar ^= 1;
  } else {
    fold_kernel<<<(c->g.ncell + 255) / 256, 256, 0, c->stream>>>(a);
    cudaError_t e = cudaMemsetAsync(c->acc, 0, sizeof(float4) * (size_t)c->g.npad, c->stream);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || a.fuse) return e;
  float4 *src = c->mtmp, *dst = c->mhalf;
  if (c->filter_on) {
    // learned filter (gated binomial fallback) on the folded deposit
    e = launch_filter(c, c->filt, c->mtmp, c->mhalf);
    if (e != cudaSuccess) return e;
    src = c->mhalf;
  } else {
    e = smooth_grid(c, src, dst, passes, &src);
    if (e != cudaSuccess) return e;
  }
  c->launches++;
  extrap_kernel<<<nb, 256, 0, c->stream>>>(c->g.ncell, src, c->mprev, c->mprev, c->mext, init);
  return cudaGetLastError();
}

cudaError_t launch_field_stage(hv_ctx *c, const float4 *Bin, const float4 *Bbase, float4 *Bout,
                               float coef) {
  StageArgs a;
  a.g = c->g;
  a.k = field_consts(c);
  a.Bin = Bin;
  a.Bbase = Bbase;
  a.Bout = Bout;
  a.mom = c->mprev;
  a.coef = coef;
  a.EB = nullptr;
  a.pin = a.pbase = nullptr;
  a.pout = nullptr;
  a.pcoef = 0.f;
  a.B0 = c->B0ext;
  c->launches++;
  if (c->g.dim2) return launch_stage_t<2, 0>(c, a);
  const size_t smem = st3d::kFloats * sizeof(float);
  static std::atomic<uint64_t> attr_set{0};
  cudaError_t e = set_smem_once(stage3d_kernel, smem, attr_set);
  if (e != cudaSuccess) return e;
  const Geom &g = c->g;
  const int blocks = ((g.nx + st3d::X - 1) / st3d::X) * ((g.ny + st3d::Y - 1) / st3d::Y) *
                     ((g.nz + st3d::Z - 1) / st3d::Z);
  return launch_pdl(stage3d_kernel, blocks, st3d::kThreads, smem, c->stream, a);
}

bool fused_substeps(const hv_ctx *c) { return c->g.dim2 != 0 && !c->g.any_open; }

cudaError_t launch_substep(hv_ctx *c, const float4 *Bin, float4 *Bout, float h) {
  SubArgs a;
  a.B0 = c->B0ext;
  a.g = c->g;
  a.k = field_consts(c);
  a.B = Bin;
  a.Bout = Bout;
  a.mom = c->mprev;
  a.h = h;
  const size_t smem = sub2d::kFloats * sizeof(float);
  static std::atomic<uint64_t> attr_set{0};
  cudaError_t e = set_smem_once(substep2d_kernel, smem, attr_set);
  if (e != cudaSuccess) return e;
  const int ntx = (c->g.nx + sub2d::SX - 1) / sub2d::SX;
  const int ntz = (c->g.nz + sub2d::SZ - 1) / sub2d::SZ;
  c->launches++;
  return launch_pdl(substep2d_kernel, ntx * ntz, kSubThreads, smem, c->stream, a);
}

// Self-consistent field smoothing (Sec. 2.2): the push gathers S^p E and
// S^p B, S being the binomial pass the moments are smoothed with, from a
// second padded array; E and B themselves stay unsmoothed.  The interior of
// the gather array is unpacked, smoothed p times and packed back with its
// ghost images.
__global__ void __launch_bounds__(256) eb_unpad_kernel(Geom g, const float4 *EB, float4 *ea,
                                                       float4 *eb) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, c, i, j, k);
    const int p = voxel_of(g, i, j, k);
    ea[c] = EB[2 * p];
    eb[c] = EB[2 * p + 1];
  }
}

__global__ void __launch_bounds__(256) eb_pad_kernel(Geom g, const float4 *ea, const float4 *eb,
                                                     float4 *EB) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, c, i, j, k);
    const float4 va = ea[c], vb = eb[c];
    if (single_image(g, i, j, k)) {
      const int p = voxel_of(g, i, j, k);
      EB[2 * p] = va;
      EB[2 * p + 1] = vb;
      continue;
    }
    int xs[5], ys[5], zs[5];
    const int nxs = axis_images(i, g.nx, xs);
    const int nys = g.dim2 ? 1 : axis_images(j, g.ny, ys);
    if (g.dim2) ys[0] = 0;
    const int nzs = axis_images(k, g.nz, zs);
    for (int a3 = 0; a3 < nzs; ++a3)
      for (int a2 = 0; a2 < nys; ++a2)
        for (int a1 = 0; a1 < nxs; ++a1) {
          const int p = xs[a1] + ys[a2] * g.sy + zs[a3] * g.sz;
          EB[2 * p] = va;
          EB[2 * p + 1] = vb;
        }
  }
}

static cudaError_t launch_field_smoothing(hv_ctx *c) {
  const int passes = c->p.field_smooth_passes;
  if (passes <= 0) return cudaSuccess;
  const int nb = elem_blocks(c->g.ncell);
  float4 *a0 = c->fsm[0], *a1 = c->fsm[1], *b0 = c->fsm[2], *b1 = c->fsm[3];
  eb_unpad_kernel<<<nb, 256, 0, c->stream>>>(c->g, c->EB, a0, b0);
  cudaError_t e = smooth_grid(c, a0, a1, passes, &a0);
  if (e == cudaSuccess) e = smooth_grid(c, b0, b1, passes, &b0);
  if (e != cudaSuccess) return e;
  eb_pad_kernel<<<nb, 256, 0, c->stream>>>(c->g, a0, b0, c->EBs);
  c->launches += 2;
  return cudaGetLastError();
}

// One explicit-midpoint stage of B and p_e together (electron energy
// equation): B_out = B_base - coef curl E(B_in, p_in), p_out = p_base +
// coef dp_e/dt(B_in, p_in), with the tiled stage kernel in 2D and 3D.
cudaError_t launch_field_stage_pe(hv_ctx *c, const float4 *Bin, const float4 *Bbase, float4 *Bout,
                                  const float *pin, const float *pbase, float *pout, float coef) {
  StageArgs a;
  a.g = c->g;
  a.k = field_consts(c);
  a.Bin = Bin;
  a.Bbase = Bbase;
  a.Bout = Bout;
  a.mom = c->mprev;
  a.coef = c->p.ohm_model == 1 ? 0.f : coef;  // the electrostatic model holds B
  a.EB = nullptr;
  a.pin = pin;
  a.pbase = pbase;
  a.pout = pout;
  a.pcoef = coef;
  a.B0 = c->B0ext;
  c->launches++;
  return c->g.dim2 ? launch_stage_t<2, 0, 1>(c, a) : launch_stage_t<3, 0, 1>(c, a);
}

// One explicit-midpoint stage of B alone with the tiled stage kernel (2D
// and 3D), for the Ohm's laws the fused kernels do not implement.
cudaError_t launch_field_stage_tiled(hv_ctx *c, const float4 *Bin, const float4 *Bbase,
                                     float4 *Bout, float coef) {
  StageArgs a;
  a.g = c->g;
  a.k = field_consts(c);
  a.Bin = Bin;
  a.Bbase = Bbase;
  a.Bout = Bout;
  a.mom = c->mprev;
  a.coef = coef;
  a.EB = nullptr;
  a.pin = a.pbase = nullptr;
  a.pout = nullptr;
  a.pcoef = 0.f;
  a.B0 = c->B0ext;
  c->launches++;
  if (c->g.any_open)
    return c->g.dim2 ? launch_stage_t<2, 0, 0, 1>(c, a) : launch_stage_t<3, 0, 0, 1>(c, a);
  return c->g.dim2 ? launch_stage_t<2, 0>(c, a) : launch_stage_t<3, 0>(c, a);
}

cudaError_t launch_pe_init(hv_ctx *c) {
  c->launches++;
  pe_init_kernel<<<elem_blocks(c->g.ncell), 256, 0, c->stream>>>(c->g.ncell, field_consts(c),
                                                                   c->mprev, c->pe);
  return cudaGetLastError();
}

const float4 *gather_array(const hv_ctx *c) {
  return c->p.field_smooth_passes > 0 ? c->EBs : c->EB;
}

cudaError_t launch_ohm_final(hv_ctx *c, const float4 *mom) {
  StageArgs a;
  a.g = c->g;
  a.k = field_consts(c);
  a.Bin = c->B;
  a.Bbase = c->B;
  a.Bout = nullptr;
  a.mom = mom;
  a.coef = 0.f;
  a.EB = c->EB;
  a.pin = c->pe;
  a.pbase = nullptr;
  a.pout = nullptr;
  a.pcoef = 0.f;
  a.B0 = c->B0ext;
  c->launches++;
  cudaError_t e;
  if (c->p.pe_eq)
    e = c->g.dim2 ? launch_stage_t<2, 1, 1>(c, a) : launch_stage_t<3, 1, 1>(c, a);
  else if (c->g.any_open)
    e = c->g.dim2 ? launch_stage_t<2, 1, 0, 1>(c, a) : launch_stage_t<3, 1, 0, 1>(c, a);
  else
    e = c->g.dim2 ? launch_stage_t<2, 1>(c, a) : launch_stage_t<3, 1>(c, a);
  if (e != cudaSuccess) return e;
  return launch_field_smoothing(c);
}

cudaError_t launch_diag(hv_ctx *c) {
  FieldConsts k = field_consts(c);
  c->launches += 2;
  grid_diag_kernel<<<c->grid_blocks, 256, 0, c->stream>>>(c->g, k, c->B, c->B0ext, c->mprev,
                                                          c->gridpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<kDiagBlocks, kDiagThreads, 0, c->stream>>>(
      c->gridpart, c->grid_blocks, c->pushpart, c->push_blocks * c->nspecies, c->vc,
      c->diag_blk, c->diag_count, c->diag_dev);
  return cudaGetLastError();
}

}  // namespace hv
