// Internal declarations shared by the libhv translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/hv.h"

namespace hv {

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// launch_pdl may be scheduled while the previous kernel of its stream is
// still draining.  Every kernel of the step calls pdl_begin() first: it
// lets the next kernel be scheduled once all of its own blocks have
// started, and waits until the previous kernel has completed and its
// memory is visible, before touching anything.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem,
                              cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Raise a kernel's dynamic shared-memory limit to `bytes` once per device:
// the attribute belongs to the device that is current when it is set, so
// `done` keeps one bit per device ordinal (ordinals above 63 set it on every
// call).
template <typename Kern>
inline cudaError_t set_smem_once(Kern kern, size_t bytes, std::atomic<uint64_t> &done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load() & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit);
  return e;
}

constexpr int kMaxSpecies = 8;

// QS deposit in the x-z layout accumulates, per cell and channel
// (n, Jx, Jy, Jz), the sums of s, s dx, s dx^2, s dz, s dz^2 (s = q w / V_c,
// times v for J); the stencil of Eq. 17 is applied to these records when
// the moments are folded onto the grid.
constexpr int kMono = 20;
// blocks of the diagnostics' final fixed-order sums
constexpr int kDiagBlocks = 64;
// diagnostics that may be pending at once (hv_diag_async)
constexpr int kDiagQueue = 4;
struct DiagSlot {
  double d[8];   // W_K, Px, Py, Pz, charge, W_B, max_divB
  int word;      // device error word
  int pad;
  int64_t step;  // the step the diagnostics describe
};

// Device error bits latched by kernels (atomicOr into the error word).
constexpr int kErrCfl = 1;     // a particle moved more than one cell in a step
constexpr int kErrNonFinite = 2;
constexpr int kErrIndex = 4;    // a corrupt cell index was skipped
constexpr int kErrTimeout = 8;  // a bounded device wait gave up

// Exact unsigned division of 32-bit values by an invariant divisor:
// q = floor(M * n / 2^64) with M = ceil(2^64 / d) (Lemire, Kaser and Kurz,
// "Faster remainder by direct computation", 2019), valid for all 32-bit n.
struct FastDiv {
  unsigned long long M;
  uint32_t d;
};

inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.M = d <= 1 ? 0ull : (~0ull / d + 1ull);
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f) {
  return f.d <= 1 ? n : (uint32_t)__umul64hi(f.M, (unsigned long long)n);
}

// Geometry of the ghost-padded gather/deposit grids.  Every axis carries
// kGhost = 2 ghost layers on each side, so a particle's voxel index
// (the padded linear index of its cell, as VPIC stores it) can move by one
// cell at the half step and still address its whole deposit stencil without
// any wrap: p = (i+2) + SY*(j+2) + SZ*(k+2).  In the 2D (x-z) layout the y
// axis is not padded: p = (i+2) + SZ*(k+2).  A ghost voxel stands for the
// interior cell ((P-2) mod n) on each axis.
constexpr int kGhost = 2;

struct Geom {
  int nx, ny, nz;
  int px, py, pz;       // padded extents (2D: py = 1)
  int sy, sz;           // padded strides (x stride is 1)
  int ncell;            // interior cells
  int npad;             // padded cells
  int dim2;             // 1: x-z plane layout (ny == 1)
  int vlo, vhi;         // voxel indices in [vlo, vhi) address their whole
                        // gather/deposit neighbourhood inside the grid
  FastDiv div_nx, div_ny;
  FastDiv div_px, div_py;  // voxel -> padded coordinates
  // supercell tiles: ions are kept sorted tile-major (tile index, then the
  // cell inside the tile), and one block of the push works on one tile
  int tx, ty, tz;       // tile extents in cells (2D: ty = 1)
  int ntx, nty, ntz;    // tiles per axis
  int ntiles;
  int tlog;             // log2(cells per tile)
  int open[3];          // 1: the axis has open faces (Sec. 2.3), 0: periodic
  int any_open;
  // sort keys predict the ion's cell kSortHorizon * sort_every / 2 steps
  // ahead: that displacement in offset units per unit velocity,
  // kSortHorizon * sort_every * dt / Delta per axis (0 on single-cell axes,
  // with open faces and without sorting: the ion's own cell)
  float pcx, pcy, pcz;
};

// Voxel index of an ion that left through an open face: it stays in its slot,
// is skipped by the push and is sorted behind the live ions.
constexpr int kDeadVox = -1;
// Error bit: injection found no free particle slot (hv_reserve_ions).
constexpr int kErrCapacity = 16;

// How far ahead the sort key predicts an ion's cell, in half sort intervals:
// 1.375 * sort_every / 2 steps.  Half an interval centres the drift on the
// interval; the push over an interval of 8 was fastest at 1.375 (measured
// 1, 1.125, 1.25, 1.375, 1.5), where it spends alike on ions that have not
// yet reached their key cell and on ions that have passed it.
#ifndef HV_SORT_HORIZON
#define HV_SORT_HORIZON 1.375
#endif
constexpr double kSortHorizon = HV_SORT_HORIZON;

// Tile extents of the supercell order: 16x16 cells in the x-z layout,
// 8x8x8 cells in 3D (cells per tile a power of two).
constexpr int kTile2X = 16, kTile2Z = 16, kTile3 = 8;
// push blocks per supercell tile
#ifndef HV_PUSH_SPLIT
#define HV_PUSH_SPLIT 2
#endif
constexpr int kPushSplit = HV_PUSH_SPLIT;

// Supercell sort key of interior cell (i, j, k): tile index, then the cell
// inside the tile, both x fastest.
__host__ __device__ __forceinline__ int supercell_key(const Geom &g, int i, int j, int k) {
  const int ti = i / g.tx, tj = j / g.ty, tk = k / g.tz;
  const int li = i - ti * g.tx, lj = j - tj * g.ty, lk = k - tk * g.tz;
  const int tile = ti + g.ntx * (tj + g.nty * tk);
  return (tile << g.tlog) + li + g.tx * (lj + g.ty * lk);
}

__host__ __device__ __forceinline__ int voxel_of(const Geom &g, int i, int j, int k) {
  return (i + kGhost) + (g.dim2 ? 0 : (j + kGhost) * g.sy) + (k + kGhost) * g.sz;
}

// Cell shift of the sort key along one axis: +1 or -1 when the offset plus
// the velocity times pc (the predicted displacement) leaves [-1, 1), else 0
// (at most one cell).  The product and the sum are rounded separately (no
// fused multiply-add), so the key is a reproducible FP32 function of the
// stored state.
__device__ __forceinline__ int pred_shift(float off, float v, float pc) {
  const float q = __fadd_rn(off, __fmul_rn(v, pc));
  return (q >= 1.f) - (q < -1.f);
}

// c + s (|s| <= 1) periodically on an axis of n cells
__host__ __device__ __forceinline__ int wrap1(int c, int n) {
  return c < 0 ? c + n : (c >= n ? c - n : c);
}

// Supercell sort key of an ion from its voxel index and its predicted cell
// shift (tile extents are powers of two).  A voxel that is not an interior
// cell gets the last key, so a corrupt index stays inside the count arrays
// (the push reports it).
__device__ __forceinline__ int ion_key(const Geom &g, int vox, int sx, int sy, int sz) {
  const int last = (g.ntiles << g.tlog) - 1;
  if (vox < g.vlo || vox >= g.vhi) return last;
  const uint32_t v = (uint32_t)vox;
  const uint32_t q = fdiv(v, g.div_px);
  int i = (int)(v - q * (uint32_t)g.px) - kGhost;
  int j = 0, k;
  if (g.dim2) {
    k = (int)q - kGhost;
  } else {
    const int kp = (int)fdiv(q, g.div_py);
    j = (int)q - kp * g.py - kGhost;
    k = kp - kGhost;
  }
  if ((unsigned)i >= (unsigned)g.nx || (unsigned)j >= (unsigned)g.ny ||
      (unsigned)k >= (unsigned)g.nz)
    return last;
  i = wrap1(i + sx, g.nx);
  j = wrap1(j + sy, g.ny);
  k = wrap1(k + sz, g.nz);
  const int lx = __ffs(g.tx) - 1, ly = __ffs(g.ty) - 1, lz = __ffs(g.tz) - 1;
  const int tile = (i >> lx) + g.ntx * ((j >> ly) + g.nty * (k >> lz));
  const int local = (i & (g.tx - 1)) + ((j & (g.ty - 1)) << lx) + ((k & (g.tz - 1)) << (lx + ly));
  return (tile << g.tlog) + local;
}

// Padded coordinates standing for interior coordinate i on an axis of n
// cells: P in [0, n + 2*kGhost) with (P - kGhost) mod n == i.  At most 5.
// True when interior cell (i, j, k) has no ghost image: it lies at least
// kGhost cells from every face (2D: along x and z).
__host__ __device__ __forceinline__ bool single_image(const Geom &g, int i, int j, int k) {
  return i >= kGhost && i < g.nx - kGhost && k >= kGhost && k < g.nz - kGhost &&
         (g.dim2 || (j >= kGhost && j < g.ny - kGhost));
}

__host__ __device__ __forceinline__ int axis_images(int i, int n, int *out) {
  int c = 0;
  const int hi = n + 2 * kGhost;
  for (int P = (i + kGhost) % n; P < hi; P += n)
    if (P >= 0) out[c++] = P;
  return c;
}

// Padded voxels whose deposits belong to interior coordinate i: the
// periodic images, or on an open axis the cell itself plus, next to a face,
// the ghost layers beyond it (deposits beyond an open face fold onto the
// cell next to it).
__host__ __device__ __forceinline__ int axis_sources(int i, int n, int open, int *out) {
  if (!open) return axis_images(i, n, out);
  int c = 0;
  out[c++] = i + kGhost;
  if (i == 0) {
    out[c++] = 0;
    out[c++] = 1;
  }
  if (i == n - 1) {
    out[c++] = n + kGhost;
    out[c++] = n + kGhost + 1;
  }
  return c;
}

// Padded voxels that hold interior coordinate i in the gather array: the
// periodic images, or on an open axis the cell itself only (the ghost layer
// holds the ghost cell's own E).
__host__ __device__ __forceinline__ int axis_holders(int i, int n, int open, int *out) {
  if (!open) return axis_images(i, n, out);
  out[0] = i + kGhost;
  return 1;
}

// Particle SoA for one species, one buffer set.  Arrays are 256-byte aligned
// and have capacity rounded up to a multiple of 4 elements.
struct Soa {
  int32_t *cell;
  float *ox, *oy, *oz;  // oy == nullptr in the 2D layout
  float *vx, *vy, *vz;
  float *w;
};

struct Species {
  double q, m;
  int64_t n, cap;
  int *tile_off;        // [ntiles + 1] first ion of each tile in the live
                        // buffer (valid ranges even before the first sort)
  int *tile_off_next;   // [ntiles + 1] the ranges the next sort writes
  int32_t *bucket;      // step sort: key counts (then offsets), scan sums
  size_t bucket_bytes;  // and every ion's rank in its key
  int32_t *wcnt;        // windowed sort: per tile and window slot, the count
  size_t wcnt_bytes;    // and then the prefix over earlier tiles
  int *n_used;          // open faces: slots in use on the device (live ions
                        // and dead slots not yet sorted out, then injected
                        // ions); n is then the slot capacity
  Soa buf[2];
  int cur;              // index of the live buffer set
  void *base[2];        // allocation bases
  size_t bytes[2];
};

struct PushConsts {
  float qmdt2;          // (q/m) dt / 2
  float cx, cy, cz;     // dt / Delta per axis (0 for single-cell axes)
  float qvc;            // q / V_c
  float ic2;            // 1 / c^2 (relativistic push only)
  double mass_d;        // m, applied to the FP64 energy and momentum sums
};

struct SortScratch;

// A drifting Maxwellian injected through an open face (face 0 -x, 1 +x, 2 -y,
// 3 +y, 4 -z, 5 +z): density n, flow u, temperature T, ion weight w.
struct InjectFace {
  int species, face;
  double n, u[3], T, w;
};

// Learned moment filter: packed bf16 weights (W1 [16][48], W2 [16][144],
// W3 [8][144], B matrices stored [n][K]), biases b1[16] b2[16] b3[8], channel
// scales and the gate thresholds.
constexpr int kFilterParams = 3492;
struct FilterParams {
  __nv_bfloat16 *w;
  float *bias;
  float scale[4];
  float nmin, rmax;
};

}  // namespace hv

struct hv_ctx {
  hv_params p;
  hv::Geom g;
  cudaStream_t stream;
  cudaStream_t side;    // a sort issued ahead of its step runs here, beside
                        // the previous step's field advance
  cudaEvent_t ev_push, ev_sort;
  cudaEvent_t ev_fold, ev_rec[2];  // QS records: a fold issued; buffer b cleared
  int rec_pending[2];   // a clear of record buffer b is issued on `side`
                        // and the next push into b has not waited for it
  int presorted;        // the current step's sort was issued on `side`
  int since_sort;       // pushes since the last sort (-1: the ions are in
                        // load order, not sorted yet)
  hv::InjectFace inject[6 * hv::kMaxSpecies];  // injection through open faces
  int ninject;
  int *inj_scratch;     // per face cell counts and offsets of an injection
  int inj_cells;
  int device;
  double vc;
  // grids (device)
  float4 *EB;           // padded [npad][2]: {Ex,Ey,Ez,Bx},{By,Bz,0,0}
  float4 *EBs;          // the same, field-smoothed, gathered by the push when
                        // field_smooth_passes > 0 (else null)
  float4 *fsm[4];       // interior [ncell] scratch of the field smoothing
  float4 *acc;          // padded [npad] per-cell deposit {n,Jx,Jy,Jz}
  float *accm[2];       // padded [npad][kMono] per-cell moment records
                        // (QS in the x-z layout), used alternately
  int accpar;           // record buffer the next deposit writes
  int filter_on;        // learned filter replaces the binomial smoothing
  hv::FilterParams filt;
  // filter training state: FP32 master parameters, Adam moments, gradient,
  // transposed bf16 weights for the backward pass
  float *tr_P, *tr_m1, *tr_m2, *tr_grad;
  __nv_bfloat16 *tr_wt;
  double *tr_loss;
  int tr_step;
  float4 *B, *Bs;       // interior [ncell] {Bx,By,Bz,0}; B1 when an external
                        // field is set
  float4 *B0ext;        // interior [ncell] fixed external field B0 of the
                        // B = B0 + B1 split (Sec. 2.3), or null
  float *pe, *pes;      // interior [ncell] electron pressure and its stage
                        // value (pe_eq = 1 only, else null)
  float4 *mhalf, *mext, *mprev, *mtmp;  // interior moments {n,Jx,Jy,Jz}
  double *pushpart;     // [kMaxSpecies][push_blocks][4]
  double *gridpart;     // [grid_blocks][4]
  double *diag_dev;     // [8]
  double *diag_blk;     // [kDiagBlocks][8] block results of the final sums
  unsigned *diag_count; // blocks of the final sums done (rearmed to 0)
  // diagnostics enqueued by hv_diag_async, oldest first: results copied to
  // page-locked host slots, an event per slot
  hv::DiagSlot *dq_host;
  cudaEvent_t dq_ev[hv::kDiagQueue];
  int dq_head, dq_count;
  int *err;             // device error word
  int push_blocks, grid_blocks;
  hv::Species sp[hv::kMaxSpecies];
  int nspecies;
  int64_t step;
  int started;
  // sort scratch (lazily sized to the largest species)
  hv::SortScratch *sort;
  // profiling
  int prof_on;
  hv_prof_t prof;
  int64_t launches;
  // allocations to release
  void *allocs[64];
  size_t alloc_bytes[64];
  int nallocs;
};

namespace hv {

// error reporting (thread-local message)
hv_status fail(hv_status s, const std::string &msg);
hv_status cuda_fail(cudaError_t e, const char *what);

// device memory through the allocation hook
void *dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void *p, size_t bytes, cudaStream_t s);

// injection through open faces (Sec. 2.3), after the push of a step
cudaError_t launch_injection(hv_ctx *c, const InjectFace &f);

// kernels launchers (return cudaGetLastError of the launch)
cudaError_t launch_push(hv_ctx *c, int species, int mode);
cudaError_t launch_moments(hv_ctx *c, int init);
bool uses_records(const hv_ctx *c);
cudaError_t launch_field_stage(hv_ctx *c, const float4 *Bin, const float4 *Bbase, float4 *Bout,
                               float coef);
cudaError_t launch_ohm_final(hv_ctx *c, const float4 *mom);
cudaError_t launch_field_stage_pe(hv_ctx *c, const float4 *Bin, const float4 *Bbase, float4 *Bout,
                                  const float *pin, const float *pbase, float *pout, float coef);
cudaError_t launch_pe_init(hv_ctx *c);
cudaError_t launch_field_stage_tiled(hv_ctx *c, const float4 *Bin, const float4 *Bbase,
                                     float4 *Bout, float coef);
const float4 *gather_array(const hv_ctx *c);
// learned moment filter (x-z layout)
cudaError_t launch_filter(hv_ctx *c, const FilterParams &fp, const float4 *in, float4 *out);
void pack_filter(const float *P, std::vector<__nv_bfloat16> &w, std::vector<float> &bias);
int filter_weight_count();
size_t filter_train_weight_count();
void pack_filter_transposed(const float *P, std::vector<__nv_bfloat16> &wt);
cudaError_t launch_filter_grad(hv_ctx *c, const FilterParams &fp, const __nv_bfloat16 *wt,
                               const float4 *m, const float4 *tg, int nbatch, float *grad,
                               double *loss);
cudaError_t launch_adam(hv_ctx *c, float *P, float *grad, float *m1, float *m2, int t, float lr,
                        const FilterParams &fp, __nv_bfloat16 *wt);
cudaError_t launch_interleave4(hv_ctx *c, int nb, const float *in, float4 *out);
// whole explicit-midpoint substeps fused in one kernel (x-z layout)
bool fused_substeps(const hv_ctx *c);  // (not with open faces)
cudaError_t launch_substep(hv_ctx *c, const float4 *Bin, float4 *Bout, float h);
cudaError_t launch_diag(hv_ctx *c);
int grid_reduce_blocks(int device);

// Stable counting sort of species s by supercell key on stream st, into the
// other buffer set (the scratch is allocated on the first call).  The
// windowed path is taken when every ion can have moved at most
// sort_window(c) cells per axis since the last sort; otherwise the general
// radix path.
hv_status sort_species(hv_ctx *c, int s, cudaStream_t st);
int sort_window(const hv_ctx *c);
// equal split of species s into tile ranges (used before the first sort)
cudaError_t tile_ranges_even(hv_ctx *c, int s);
void sort_release(hv_ctx *c);
// standalone key sort into perm with scratch from the allocation hook
hv_status sort_keys(const int32_t *keys, int64_t n, int32_t nkeys, int32_t *perm,
                    int32_t *counts, cudaStream_t stream, int64_t *launches);

}  // namespace hv
