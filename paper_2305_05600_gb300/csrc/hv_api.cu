// C ABI of libhv: argument checks, device state, and the order of kernels in
// one step of the hybrid PIC ion loop (Sec. 2.2 of the paper):
//   [sort] -> push/gather/deposit -> moment post (fold, smoothing, Eq. 11)
//   -> nsub x 2 Ohm/Faraday stages (Eq. 5, explicit midpoint) -> final Ohm.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hv_internal.cuh"

namespace {

thread_local std::string g_err = "no error";
hv_alloc_fn g_alloc = nullptr;
hv_free_fn g_free = nullptr;
void *g_user = nullptr;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

namespace hv {

hv_status fail(hv_status s, const std::string &msg) {
  g_err = msg;
  return s;
}

hv_status cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? HV_ENOMEM : HV_ECUDA;
}

void *dev_alloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 256;
  if (g_alloc) return g_alloc(bytes, (void *)s, g_user);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void *p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (bytes == 0) bytes = 256;
  if (g_free) {
    g_free(p, bytes, (void *)s, g_user);
    return;
  }
  cudaFreeAsync(p, s);
}

}  // namespace hv

using namespace hv;

namespace {

void *ctx_alloc(hv_ctx *c, size_t bytes) {
  if (c->nallocs >= 64) return nullptr;
  void *p = dev_alloc(bytes, c->stream);
  if (p) {
    c->allocs[c->nallocs] = p;
    c->alloc_bytes[c->nallocs] = bytes;
    c->nallocs++;
  }
  return p;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

hv_status check_params(const hv_params *p) {
  if (!p) return fail(HV_EINVAL, "params is NULL");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(HV_EINVAL, "nx, ny, nz must be >= 1");
  if ((int64_t)p->nx * p->ny * p->nz >= ((int64_t)1 << 31) ||
      (int64_t)(p->nx + 2) * (p->ny + 2) * (p->nz + 2) >= ((int64_t)1 << 30))
    return fail(HV_EINVAL, "grid too large (cell indices are int32)");
  if (p->nsub < 1) return fail(HV_EINVAL, "nsub must be >= 1");
  {
    const int64_t tx = p->ny == 1 ? kTile2X : kTile3, ty = p->ny == 1 ? 1 : kTile3;
    const int64_t tz = p->ny == 1 ? kTile2Z : kTile3;
    const int64_t nt = ((p->nx + tx - 1) / tx) * ((p->ny + ty - 1) / ty) * ((p->nz + tz - 1) / tz);
    if (nt * tx * ty * tz >= ((int64_t)1 << 31))
      return fail(HV_EINVAL, "grid too large for int32 supercell keys");
  }
  if (!finite_pos(p->dx) || !finite_pos(p->dy) || !finite_pos(p->dz) || !finite_pos(p->dt))
    return fail(HV_EINVAL, "dx, dy, dz, dt must be finite and > 0");
  if (!std::isfinite(p->Te) || p->Te < 0) return fail(HV_EINVAL, "Te must be finite and >= 0");
  if (!finite_pos(p->gamma_e)) return fail(HV_EINVAL, "gamma_e must be > 0");
  if (!std::isfinite(p->eta) || p->eta < 0 || !std::isfinite(p->eta_h) || p->eta_h < 0)
    return fail(HV_EINVAL, "eta and eta_h must be finite and >= 0");
  if (!finite_pos(p->n_floor)) return fail(HV_EINVAL, "n_floor must be > 0 (Ohm's law divides by n)");
  if (p->shape < 0 || p->shape > 2) return fail(HV_EINVAL, "shape must be 0 (NGP), 1 (QS) or 2 (CIC)");
  if (p->smooth_passes < 0 || p->smooth_passes > 64) return fail(HV_EINVAL, "smooth_passes in [0, 64]");
  if (p->sort_every < 0) return fail(HV_EINVAL, "sort_every must be >= 0");
  if (p->field_smooth_passes < 0 || p->field_smooth_passes > 64)
    return fail(HV_EINVAL, "field_smooth_passes in [0, 64]");
  if (p->pe_eq != 0 && p->pe_eq != 1) return fail(HV_EINVAL, "pe_eq must be 0 or 1");
  if (p->ohm_model < 0 || p->ohm_model > 2) return fail(HV_EINVAL, "ohm_model must be 0, 1 or 2");
  if (p->relativistic != 0 && p->relativistic != 1)
    return fail(HV_EINVAL, "relativistic must be 0 or 1");
  if (p->relativistic && !finite_pos(p->c_light))
    return fail(HV_EINVAL, "c_light must be finite and > 0 for the relativistic push");
  if (p->open_faces & ~7) return fail(HV_EINVAL, "open_faces takes bits 1 (x), 2 (y), 4 (z)");
  if (p->open_faces) {
    const int32_t n3[3] = {p->nx, p->ny, p->nz};
    for (int a = 0; a < 3; ++a)
      if ((p->open_faces >> a & 1) && n3[a] < 2)
        return fail(HV_EINVAL, "an open axis needs more than one cell");
    if (p->ohm_model != 0 || p->pe_eq || p->smooth_passes || p->field_smooth_passes ||
        p->relativistic)
      return fail(HV_EINVAL, "open faces are built for the hybrid Ohm's law with the equation "
                             "of state, without smoothing and without the relativistic push");
  }
  if (!std::isfinite(p->kappa) || p->kappa < 0) return fail(HV_EINVAL, "kappa must be finite and >= 0");
  if (p->pe_eq && p->kappa > 0) {
    // explicit heat conduction at the density floor: the explicit-midpoint
    // step is stable for h (gamma - 1) kappa / n_floor * sum 4 / Delta^2 <= 2
    double s2 = 0;
    if (p->nx > 1) s2 += 4.0 / (p->dx * p->dx);
    if (p->ny > 1) s2 += 4.0 / (p->dy * p->dy);
    if (p->nz > 1) s2 += 4.0 / (p->dz * p->dz);
    const double r = p->dt / p->nsub * (p->gamma_e - 1.0) * p->kappa / p->n_floor * s2;
    if (r > 2.0) {
      char buf[160];
      snprintf(buf, sizeof buf, "heat-conduction limit violated: h (gamma-1) kappa / n_floor * "
               "sum 4/dx^2 = %g > 2", r);
      return fail(HV_ECFL, buf);
    }
  }
  // whistler limit Omega_ci h < Delta^2 / pi (Sec. 2.1) for the field step h
  double dmin = 1e300;
  if (p->nx > 1) dmin = std::fmin(dmin, p->dx);
  if (p->ny > 1) dmin = std::fmin(dmin, p->dy);
  if (p->nz > 1) dmin = std::fmin(dmin, p->dz);
  if (p->ohm_model == 2 && p->eta > 0) {
    // resistive diffusion of B: the explicit-midpoint step is stable for
    // h eta sum 4 / Delta^2 <= 2 (centred curl of curl: sin^2 <= 1)
    double s2 = 0;
    if (p->nx > 1) s2 += 4.0 / (p->dx * p->dx);
    if (p->ny > 1) s2 += 4.0 / (p->dy * p->dy);
    if (p->nz > 1) s2 += 4.0 / (p->dz * p->dz);
    const double r = p->dt / p->nsub * p->eta * s2;
    if (r > 2.0) {
      char buf[160];
      snprintf(buf, sizeof buf, "resistive diffusion limit violated: h eta sum 4/dx^2 = %g > 2", r);
      return fail(HV_ECFL, buf);
    }
  }
  // (only the hybrid Ohm's law has the Hall term and its whistler)
  if (p->ohm_model == 0 && dmin < 1e300 && p->dt / p->nsub >= dmin * dmin / M_PI) {
    char buf[160];
    snprintf(buf, sizeof buf, "whistler limit violated: dt/nsub = %g >= dx^2/pi = %g",
             p->dt / p->nsub, dmin * dmin / M_PI);
    return fail(HV_ECFL, buf);
  }
  return HV_OK;
}

Geom make_geom(const hv_params *p) {
  Geom g;
  g.nx = p->nx;
  g.ny = p->ny;
  g.nz = p->nz;
  g.dim2 = p->ny == 1;
  g.px = p->nx + 2 * kGhost;
  g.py = g.dim2 ? 1 : p->ny + 2 * kGhost;
  g.pz = p->nz + 2 * kGhost;
  g.sy = g.px;
  g.sz = g.px * g.py;
  g.ncell = p->nx * p->ny * p->nz;
  g.npad = g.px * g.py * g.pz;
  g.vlo = 2 * (1 + (g.dim2 ? 0 : g.sy) + g.sz);
  g.vhi = g.npad - g.vlo;
  g.div_nx = make_fastdiv((uint32_t)p->nx);
  g.div_ny = make_fastdiv((uint32_t)p->ny);
  g.div_px = make_fastdiv((uint32_t)g.px);
  g.div_py = make_fastdiv((uint32_t)g.py);
  g.tx = g.dim2 ? kTile2X : kTile3;
  g.ty = g.dim2 ? 1 : kTile3;
  g.tz = g.dim2 ? kTile2Z : kTile3;
  g.ntx = (p->nx + g.tx - 1) / g.tx;
  g.nty = (p->ny + g.ty - 1) / g.ty;
  g.ntz = (p->nz + g.tz - 1) / g.tz;
  g.ntiles = g.ntx * g.nty * g.ntz;
  g.tlog = 0;
  while ((1 << g.tlog) < g.tx * g.ty * g.tz) ++g.tlog;
  for (int a = 0; a < 3; ++a) g.open[a] = (p->open_faces >> a) & 1;
  g.any_open = p->open_faces != 0;
  const bool pred = p->sort_every > 0 && !g.any_open;
  g.pcx = pred && p->nx > 1 ? (float)(kSortHorizon * p->sort_every * p->dt / p->dx) : 0.f;
  g.pcy = pred && p->ny > 1 ? (float)(kSortHorizon * p->sort_every * p->dt / p->dy) : 0.f;
  g.pcz = pred && p->nz > 1 ? (float)(kSortHorizon * p->sort_every * p->dt / p->dz) : 0.f;
  return g;
}

__host__ __device__ int voxel_to_linear(const Geom &g, int v) {
  const int k = v / g.sz - kGhost;
  const int r = v % g.sz;
  const int j = g.dim2 ? 0 : r / g.sy - kGhost;
  const int i = (g.dim2 ? r : r % g.sy) - kGhost;
  return i + g.nx * (j + g.ny * k);
}

__global__ void vox_to_linear_kernel(Geom g, const int *in, int *out, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = voxel_to_linear(g, in[t]);
}

// Check loaded ions and convert them in place: cell index -> voxel index,
// relative coordinates along single-cell axes -> 0.  Bits of *bad: 1 bad
// cell, 2 bad offset, 4 non-finite velocity or weight.
__global__ void load_check_kernel(Geom g, Soa s, int64_t n, int *bad) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int c = s.cell[t];
    int flag = 0;
    if (c < 0 || c >= g.ncell) {
      flag |= 1;
      s.cell[t] = g.vlo;  // keep the array valid for the (discarded) buffer
    } else {
      const int i = c % g.nx, j = (c / g.nx) % g.ny, k = c / (g.nx * g.ny);
      s.cell[t] = voxel_of(g, i, j, k);
    }
    float *o[3] = {s.ox, s.oy, s.oz};
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
      if (!o[a]) continue;
      if (nn[a] == 1) {
        o[a][t] = 0.f;
      } else {
        const float v = o[a][t];
        if (!(v >= -1.f && v < 1.f)) flag |= 2;
      }
    }
    if (!isfinite(s.vx[t]) || !isfinite(s.vy[t]) || !isfinite(s.vz[t]) || !isfinite(s.w[t]))
      flag |= 4;
    if (flag) atomicOr(bad, flag);
  }
}

// component-major [3][ncell] <-> interleaved float4 grids, and the padded
// gather array's E part
__global__ void unpack4_kernel(int ncell, const float4 *in, int ncomp, int first, float *out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    const float4 v = in[c];
    const float a[4] = {v.x, v.y, v.z, v.w};
    for (int m = 0; m < ncomp; ++m) out[(size_t)m * ncell + c] = a[first + m];
  }
}

// B component-major, with the external field added back (the total field)
__global__ void unpack_B_kernel(int ncell, const float4 *B, const float4 *B0, float *out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    float4 v = B[c];
    if (B0) {
      const float4 e = B0[c];
      v = make_float4(v.x + e.x, v.y + e.y, v.z + e.z, 0.f);
    }
    out[c] = v.x;
    out[(size_t)ncell + c] = v.y;
    out[(size_t)2 * ncell + c] = v.z;
  }
}

// B1 = B - B0 when an external field is set
__global__ void sub_ext_kernel(int ncell, float4 *B, const float4 *B0) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    const float4 v = B[c], e = B0[c];
    B[c] = make_float4(v.x - e.x, v.y - e.y, v.z - e.z, 0.f);
  }
}

__global__ void unpack_E_kernel(Geom g, const float4 *EB, float *out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += gridDim.x * blockDim.x) {
    const int i = c % g.nx;
    const int j = (c / g.nx) % g.ny;
    const int k = c / (g.nx * g.ny);
    const float4 e = EB[2 * voxel_of(g, i, j, k)];
    out[c] = e.x;
    out[(size_t)g.ncell + c] = e.y;
    out[(size_t)2 * g.ncell + c] = e.z;
  }
}

int eblocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

// The status reported for a device error word (see hv_error_status).
hv_status status_of_word(int e) {
  if (e & kErrNonFinite) return fail(HV_ENAN, "a particle became non-finite");
  if (e & kErrCfl) return fail(HV_ECFL, "a particle moved more than one cell in one step");
  if (e & kErrIndex) return fail(HV_ECUDA, "a corrupt particle cell index was found");
  if (e & kErrTimeout) return fail(HV_ETIMEOUT, "a bounded device wait gave up");
  if (e & kErrCapacity)
    return fail(HV_ENOMEM, "no free particle slot for injected ions (see hv_reserve_ions)");
  return HV_OK;
}

hv_status latched(hv_ctx *c, int *word) {
  int e = 0;
  cudaError_t r = cudaMemcpyAsync(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (r == cudaSuccess) r = cudaStreamSynchronize(c->stream);
  if (r != cudaSuccess) return cuda_fail(r, "synchronise");
  if (word) *word = e;
  return status_of_word(e);
}

__global__ void inject_error_kernel(int *err, int bits) { atomicOr(err, bits); }

// Side stream and events for sorts issued ahead of their step, created on
// first use.
hv_status side_stream(hv_ctx *c) {
  if (c->side) return HV_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_push, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_sort, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fold, cudaEventDisableTiming);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    e = cudaEventCreateWithFlags(&c->ev_rec[b], cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_fail(e, "side stream");
  return HV_OK;
}

// QS moment records (x-z layout) are double-buffered: a push deposits into
// one buffer while the other waits for its next push.  The buffer the fold
// just read is cleared on the side stream, beside the field advance, and
// the push that deposits into it next waits for the clear.
hv_status clear_records_async(hv_ctx *c) {
  if (!uses_records(c)) return HV_OK;
  hv_status st = side_stream(c);
  if (st != HV_OK) return st;
  const int b = c->accpar ^ 1;  // read by the fold just issued (the fold flips accpar)
  cudaError_t e = cudaEventRecord(c->ev_fold, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->side, c->ev_fold, 0);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->accm[b], 0, sizeof(float) * kMono * (size_t)c->g.npad, c->side);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_rec[b], c->side);
  if (e != cudaSuccess) return cuda_fail(e, "record clear");
  c->rec_pending[b] = 1;
  return HV_OK;
}

void wait_records(hv_ctx *c) {
  if (!c->rec_pending[c->accpar]) return;
  cudaStreamWaitEvent(c->stream, c->ev_rec[c->accpar], 0);
  c->rec_pending[c->accpar] = 0;
}

hv_status startup(hv_ctx *c) {
  wait_records(c);
  for (int s = 0; s < c->nspecies; ++s) {
    cudaError_t e = launch_push(c, s, 1);
    if (e != cudaSuccess) return cuda_fail(e, "start-up deposit");
  }
  cudaError_t e = launch_moments(c, 1);
  if (e != cudaSuccess) return cuda_fail(e, "start-up moments");
  hv_status rs = clear_records_async(c);
  if (rs != HV_OK) return rs;
  if (c->p.pe_eq) {
    e = launch_pe_init(c);
    if (e != cudaSuccess) return cuda_fail(e, "start-up electron pressure");
  }
  e = launch_ohm_final(c, c->mext);
  if (e != cudaSuccess) return cuda_fail(e, "start-up Ohm");
  c->started = 1;
  return HV_OK;
}

// Events of one profiled step: e[0..5] bracket the phases on the context
// stream; e[6], e[7] bracket a sort issued on the side stream (side = 1),
// whose own duration is added to the sort time.
struct StepEvents {
  cudaEvent_t e[8];
  int64_t launches[5];
  int side;
};

}  // namespace

// per-context profiling records (kept outside the POD context)
namespace {
struct ProfStore {
  hv_ctx *owner;
  std::vector<StepEvents> rec;
  std::vector<cudaEvent_t> pool;
};
std::vector<ProfStore *> g_prof;

ProfStore *prof_store(hv_ctx *c, bool create) {
  for (auto *p : g_prof)
    if (p->owner == c) return p;
  if (!create) return nullptr;
  ProfStore *p = new ProfStore();
  p->owner = c;
  g_prof.push_back(p);
  return p;
}

cudaEvent_t prof_event(ProfStore *ps) {
  if (!ps->pool.empty()) {
    cudaEvent_t e = ps->pool.back();
    ps->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_recycle(ProfStore *ps) {
  for (auto &r : ps->rec)
    for (int i = 0; i < 8; ++i) ps->pool.push_back(r.e[i]);
  ps->rec.clear();
}

void prof_destroy(hv_ctx *c) {
  for (size_t i = 0; i < g_prof.size(); ++i) {
    if (g_prof[i]->owner == c) {
      prof_recycle(g_prof[i]);
      for (auto e : g_prof[i]->pool) cudaEventDestroy(e);
      delete g_prof[i];
      g_prof.erase(g_prof.begin() + i);
      return;
    }
  }
}
}  // namespace

extern "C" {

hv_status hv_set_allocator(hv_alloc_fn alloc, hv_free_fn free_fn, void *user) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(HV_EINVAL, "alloc and free hooks must be given together");
  g_alloc = alloc;
  g_free = free_fn;
  g_user = user;
  return HV_OK;
}

const char *hv_last_error(void) { return g_err.c_str(); }

hv_status hv_init_grid(const hv_params *p, const float *B0_host, void *cuda_stream,
                       hv_ctx **out) {
  if (!out) return fail(HV_EINVAL, "out is NULL");
  *out = nullptr;
  hv_status st = check_params(p);
  if (st != HV_OK) return st;
  hv_ctx *c = new hv_ctx();
  memset((void *)c, 0, sizeof(hv_ctx));
  c->p = *p;
  c->g = make_geom(p);
  c->stream = (cudaStream_t)cuda_stream;
  c->since_sort = -1;  // ions arrive in load order
  cudaGetDevice(&c->device);
  c->vc = p->dx * p->dy * p->dz;
  c->push_blocks = c->g.ntiles * kPushSplit;  // push blocks (kPushSplit per supercell tile)
  c->grid_blocks = grid_reduce_blocks(c->device);
  const Geom &g = c->g;
  const size_t npad = (size_t)g.npad, nc = (size_t)g.ncell;
  c->EB = (float4 *)ctx_alloc(c, sizeof(float4) * 2 * npad);
  c->acc = (float4 *)ctx_alloc(c, sizeof(float4) * npad);
  c->B = (float4 *)ctx_alloc(c, sizeof(float4) * nc);
  c->Bs = (float4 *)ctx_alloc(c, sizeof(float4) * nc);
  c->mhalf = (float4 *)ctx_alloc(c, sizeof(float4) * nc);
  c->mext = (float4 *)ctx_alloc(c, sizeof(float4) * nc);
  c->mprev = (float4 *)ctx_alloc(c, sizeof(float4) * nc);
  c->mtmp = (float4 *)ctx_alloc(c, sizeof(float4) * nc);
  c->pushpart = (double *)ctx_alloc(c, sizeof(double) * kMaxSpecies * c->push_blocks * 4);
  c->gridpart = (double *)ctx_alloc(c, sizeof(double) * c->grid_blocks * 4);
  c->diag_dev = (double *)ctx_alloc(c, sizeof(double) * 8);
  c->diag_blk = (double *)ctx_alloc(c, sizeof(double) * 8 * kDiagBlocks);
  c->diag_count = (unsigned *)ctx_alloc(c, sizeof(unsigned));
  c->err = (int *)ctx_alloc(c, sizeof(int));
  const bool rec = p->shape == HV_SHAPE_QS && c->g.dim2;
  for (int b = 0; b < 2; ++b)
    c->accm[b] = rec ? (float *)ctx_alloc(c, sizeof(float) * kMono * npad) : nullptr;
  if (p->pe_eq) {
    c->pe = (float *)ctx_alloc(c, sizeof(float) * nc);
    c->pes = (float *)ctx_alloc(c, sizeof(float) * nc);
  }
  const bool fsm = p->field_smooth_passes > 0;
  if (fsm) {
    c->EBs = (float4 *)ctx_alloc(c, sizeof(float4) * 2 * npad);
    for (int b = 0; b < 4; ++b) c->fsm[b] = (float4 *)ctx_alloc(c, sizeof(float4) * nc);
  }
  if (!c->EB || !c->acc || !c->B || !c->Bs || !c->mhalf || !c->mext || !c->mprev || !c->mtmp ||
      !c->pushpart || !c->gridpart || !c->diag_dev || !c->diag_blk || !c->diag_count || !c->err ||
      (rec && (!c->accm[0] || !c->accm[1])) ||
      (fsm && (!c->EBs || !c->fsm[0] || !c->fsm[1] || !c->fsm[2] || !c->fsm[3])) ||
      (p->pe_eq && (!c->pe || !c->pes))) {
    hv_destroy(c);
    return fail(HV_ENOMEM, "grid allocation failed");
  }
  cudaMemsetAsync(c->EB, 0, sizeof(float4) * 2 * npad, c->stream);
  if (fsm) cudaMemsetAsync(c->EBs, 0, sizeof(float4) * 2 * npad, c->stream);
  cudaMemsetAsync(c->acc, 0, sizeof(float4) * npad, c->stream);
  cudaMemsetAsync(c->mprev, 0, sizeof(float4) * nc, c->stream);
  cudaMemsetAsync(c->mext, 0, sizeof(float4) * nc, c->stream);
  cudaMemsetAsync(c->pushpart, 0, sizeof(double) * kMaxSpecies * c->push_blocks * 4, c->stream);
  cudaMemsetAsync(c->diag_dev, 0, sizeof(double) * 8, c->stream);
  cudaMemsetAsync(c->diag_count, 0, sizeof(unsigned), c->stream);
  cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
  for (int b = 0; b < 2; ++b)
    if (c->accm[b]) cudaMemsetAsync(c->accm[b], 0, sizeof(float) * kMono * npad, c->stream);
  std::vector<float4> hb(nc);
  for (size_t i = 0; i < nc; ++i) {
    if (B0_host) {
      hb[i] = make_float4(B0_host[i], B0_host[nc + i], B0_host[2 * nc + i], 0.f);
      if (!std::isfinite(hb[i].x) || !std::isfinite(hb[i].y) || !std::isfinite(hb[i].z)) {
        hv_destroy(c);
        return fail(HV_EINVAL, "B0 has a non-finite value");
      }
    } else {
      hb[i] = make_float4(1.f, 0.f, 0.f, 0.f);
    }
  }
  cudaError_t e = cudaMemcpyAsync(c->B, hb.data(), sizeof(float4) * nc, cudaMemcpyHostToDevice,
                                  c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    hv_destroy(c);
    return cuda_fail(e, "hv_init_grid upload");
  }
  *out = c;
  return HV_OK;
}

hv_status hv_set_external_field(hv_ctx *c, const float *B0_host) {
  if (!c || !B0_host) return fail(HV_EINVAL, "ctx or B0 is NULL");
  if (c->started) return fail(HV_ESTATE, "the external field must be set before the first step");
  if (c->B0ext) return fail(HV_ESTATE, "the external field is already set");
  const size_t nc = (size_t)c->g.ncell;
  std::vector<float4> hb(nc);
  for (size_t i = 0; i < nc; ++i) {
    hb[i] = make_float4(B0_host[i], B0_host[nc + i], B0_host[2 * nc + i], 0.f);
    if (!std::isfinite(hb[i].x) || !std::isfinite(hb[i].y) || !std::isfinite(hb[i].z))
      return fail(HV_EINVAL, "the external field has a non-finite value");
  }
  float4 *d = (float4 *)ctx_alloc(c, sizeof(float4) * nc);
  if (!d) return fail(HV_ENOMEM, "external field allocation failed");
  cudaError_t e = cudaMemcpyAsync(d, hb.data(), sizeof(float4) * nc, cudaMemcpyHostToDevice,
                                  c->stream);
  if (e == cudaSuccess) {
    sub_ext_kernel<<<eblocks(nc), 256, 0, c->stream>>>(c->g.ncell, c->B, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_set_external_field");
  c->B0ext = d;
  return HV_OK;
}

hv_status hv_load_ions(hv_ctx *c, int32_t species, double q, double m, int64_t n,
                       const int32_t *cell, const float *off3, const float *v3, const float *w,
                       int on_device) {
  if (!c) return fail(HV_EINVAL, "ctx is NULL");
  if (c->started) return fail(HV_ESTATE, "ions must be loaded before the first step");
  if (species != c->nspecies || species >= kMaxSpecies)
    return fail(HV_EINVAL, "species must be the next index (at most 8 species)");
  if (!std::isfinite(q) || !std::isfinite(m) || m <= 0 || q == 0)
    return fail(HV_EINVAL, "q must be finite and non-zero, m finite and > 0");
  if (n < 0 || n >= ((int64_t)1 << 31) - 4) return fail(HV_EINVAL, "n must be in [0, 2^31 - 4)");
  if (n > 0 && (!cell || !off3 || !v3 || !w)) return fail(HV_EINVAL, "null particle array");
  const Geom &g = c->g;
  Species &sp = c->sp[species];
  sp.q = q;
  sp.m = m;
  sp.n = n;
  sp.cap = ((n + 3) / 4) * 4;
  if (sp.cap == 0) sp.cap = 4;
  const size_t arr = align256(sizeof(float) * sp.cap);
  const int narr = g.dim2 ? 7 : 8;
  for (int b = 0; b < 2; ++b) {
    sp.bytes[b] = arr * narr;
    sp.base[b] = dev_alloc(sp.bytes[b], c->stream);
    if (!sp.base[b]) {
      if (b == 1) dev_free(sp.base[0], sp.bytes[0], c->stream);
      return fail(HV_ENOMEM, "particle allocation failed");
    }
    cudaMemsetAsync(sp.base[b], 0, sp.bytes[b], c->stream);
    char *p = (char *)sp.base[b];
    Soa &s = sp.buf[b];
    int slot = 0;
    s.cell = (int32_t *)(p + arr * slot++);
    s.ox = (float *)(p + arr * slot++);
    s.oy = g.dim2 ? nullptr : (float *)(p + arr * slot++);
    s.oz = (float *)(p + arr * slot++);
    s.vx = (float *)(p + arr * slot++);
    s.vy = (float *)(p + arr * slot++);
    s.vz = (float *)(p + arr * slot++);
    s.w = (float *)(p + arr * slot++);
  }
  sp.tile_off = (int *)dev_alloc(sizeof(int) * 2 * (g.ntiles + 1), c->stream);
  if (!sp.tile_off) {
    for (int b = 0; b < 2; ++b) dev_free(sp.base[b], sp.bytes[b], c->stream);
    return fail(HV_ENOMEM, "tile range allocation failed");
  }
  sp.tile_off_next = sp.tile_off + (g.ntiles + 1);
  sp.cur = 0;
  // copy straight from the caller's arrays, then check and convert on the
  // device (interior cell -> voxel, single-cell-axis offsets -> 0)
  cudaError_t e = cudaSuccess;
  if (n > 0) {
    Soa &s = sp.buf[0];
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t b4 = 4 * (size_t)n;
    e = cudaMemcpyAsync(s.cell, cell, b4, k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.ox, off3, b4, k, c->stream);
    if (e == cudaSuccess && s.oy) e = cudaMemcpyAsync(s.oy, off3 + n, b4, k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.oz, off3 + 2 * n, b4, k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.vx, v3, b4, k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.vy, v3 + n, b4, k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.vz, v3 + 2 * n, b4, k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.w, w, b4, k, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) {
      const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8192);
      load_check_kernel<<<blocks, 256, 0, c->stream>>>(g, s, n, c->err);
      e = cudaGetLastError();
    }
  }
  int bad = 0;
  if (e == cudaSuccess && n > 0)
    e = cudaMemcpyAsync(&bad, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && n > 0) e = cudaMemsetAsync(c->err, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess || bad) {
    for (int b = 0; b < 2; ++b) dev_free(sp.base[b], sp.bytes[b], c->stream);
    dev_free(std::min(sp.tile_off, sp.tile_off_next), sizeof(int) * 2 * (g.ntiles + 1), c->stream);
    memset(&sp, 0, sizeof(sp));
    if (e != cudaSuccess) return cuda_fail(e, "hv_load_ions upload");
    if (bad & 1) return fail(HV_EINVAL, "cell index out of range");
    if (bad & 2) return fail(HV_EINVAL, "relative coordinate outside [-1, 1) or non-finite");
    return fail(HV_EINVAL, "non-finite velocity or weight");
  }
  if (g.any_open) {
    // slots in use, counted on the device (absorption and injection change it)
    sp.n_used = (int *)ctx_alloc(c, sizeof(int));
    if (!sp.n_used) return fail(HV_ENOMEM, "slot counter allocation failed");
    const int nn = (int)n;
    e = cudaMemcpyAsync(sp.n_used, &nn, sizeof(int), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "slot counter");
  }
  c->nspecies++;
  e = tile_ranges_even(c, species);
  if (e != cudaSuccess) return cuda_fail(e, "tile ranges");
  return HV_OK;
}

__global__ void mark_dead_kernel(int32_t *cell, int64_t lo, int64_t hi) {
  for (int64_t t = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < hi;
       t += (int64_t)gridDim.x * blockDim.x)
    cell[t] = kDeadVox;
}

hv_status hv_reserve_ions(hv_ctx *c, int32_t species, int64_t capacity) {
  if (!c) return fail(HV_EINVAL, "ctx is NULL");
  if (!c->g.any_open) return fail(HV_EINVAL, "slot reserve is for contexts with open faces");
  if (c->started) return fail(HV_ESTATE, "reserve slots before the first step");
  if (species < 0 || species >= c->nspecies) return fail(HV_EINVAL, "no such species");
  Species &sp = c->sp[species];
  if (capacity < sp.n || capacity >= ((int64_t)1 << 31) - 4)
    return fail(HV_EINVAL, "capacity must be at least the loaded ions and below 2^31 - 4");
  const Geom &g = c->g;
  const int64_t cap = std::max<int64_t>(4, ((capacity + 3) / 4) * 4);
  const size_t arr = align256(sizeof(float) * cap);
  const int narr = g.dim2 ? 7 : 8;
  void *base[2] = {nullptr, nullptr};
  Soa buf[2];
  for (int b = 0; b < 2; ++b) {
    base[b] = dev_alloc(arr * narr, c->stream);
    if (!base[b]) {
      if (b) dev_free(base[0], arr * narr, c->stream);
      return fail(HV_ENOMEM, "particle allocation failed");
    }
    char *q = (char *)base[b];
    int slot = 0;
    buf[b].cell = (int32_t *)(q + arr * slot++);
    buf[b].ox = (float *)(q + arr * slot++);
    buf[b].oy = g.dim2 ? nullptr : (float *)(q + arr * slot++);
    buf[b].oz = (float *)(q + arr * slot++);
    buf[b].vx = (float *)(q + arr * slot++);
    buf[b].vy = (float *)(q + arr * slot++);
    buf[b].vz = (float *)(q + arr * slot++);
    buf[b].w = (float *)(q + arr * slot++);
  }
  const Soa &o = sp.buf[sp.cur];
  const size_t b4 = 4 * (size_t)sp.n;
  cudaError_t e = cudaSuccess;
  if (sp.n > 0) {
    const void *src[8] = {o.cell, o.ox, o.oy, o.oz, o.vx, o.vy, o.vz, o.w};
    void *dst[8] = {buf[0].cell, buf[0].ox, buf[0].oy, buf[0].oz, buf[0].vx, buf[0].vy,
                    buf[0].vz, buf[0].w};
    for (int f = 0; f < 8 && e == cudaSuccess; ++f)
      if (src[f]) e = cudaMemcpyAsync(dst[f], src[f], b4, cudaMemcpyDeviceToDevice, c->stream);
  }
  if (e == cudaSuccess && cap > sp.n) {
    mark_dead_kernel<<<eblocks(cap - sp.n), 256, 0, c->stream>>>(buf[0].cell, sp.n, cap);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    for (int b = 0; b < 2; ++b) dev_free(base[b], arr * narr, c->stream);
    return cuda_fail(e, "hv_reserve_ions");
  }
  for (int b = 0; b < 2; ++b) dev_free(sp.base[b], sp.bytes[b], c->stream);
  for (int b = 0; b < 2; ++b) {
    sp.base[b] = base[b];
    sp.bytes[b] = arr * narr;
    sp.buf[b] = buf[b];
  }
  sp.cur = 0;
  sp.cap = cap;
  sp.n = cap;  // slots; the device counter keeps the ones in use
  if (sp.bucket) {  // sized for the old slot count
    dev_free(sp.bucket, sp.bucket_bytes, c->stream);
    sp.bucket = nullptr;
  }
  return HV_OK;
}

hv_status hv_set_injection(hv_ctx *c, int32_t species, int32_t face, double n, const double *u,
                           double T, double w) {
  if (!c || !u) return fail(HV_EINVAL, "ctx or u is NULL");
  if (c->started) return fail(HV_ESTATE, "set injection before the first step");
  if (species < 0 || species >= c->nspecies) return fail(HV_EINVAL, "no such species");
  if (face < 0 || face > 5 || !c->g.open[face / 2])
    return fail(HV_EINVAL, "face must be 0..5 on an axis with open faces");
  if (!std::isfinite(n) || n < 0 || !std::isfinite(T) || T < 0 || !std::isfinite(w) || w <= 0 ||
      !std::isfinite(u[0]) || !std::isfinite(u[1]) || !std::isfinite(u[2]))
    return fail(HV_EINVAL, "n, T >= 0, w > 0 and u must be finite");
  if (c->ninject >= 6 * kMaxSpecies) return fail(HV_EINVAL, "too many injection faces");
  InjectFace f;
  f.species = species;
  f.face = face;
  f.n = n;
  f.T = T;
  f.w = w;
  for (int a = 0; a < 3; ++a) f.u[a] = u[a];
  const int n3[3] = {c->g.nx, c->g.ny, c->g.nz};
  const int ax = face / 2;
  const int cells = n3[(ax + 1) % 3] * n3[(ax + 2) % 3];
  if (cells + 1 > c->inj_cells) {
    int *q = (int *)ctx_alloc(c, sizeof(int) * (size_t)(cells + 1));
    if (!q) return fail(HV_ENOMEM, "injection scratch allocation failed");
    c->inj_scratch = q;
    c->inj_cells = cells + 1;
  }
  c->inject[c->ninject++] = f;
  return HV_OK;
}

hv_status hv_step(hv_ctx *c, int32_t nsteps) {
  if (!c) return fail(HV_EINVAL, "ctx is NULL");
  if (nsteps < 0) return fail(HV_EINVAL, "nsteps must be >= 0");
  if (!c->started) {
    hv_status st = startup(c);
    if (st != HV_OK) return st;
  }
  ProfStore *ps = c->prof_on ? prof_store(c, true) : nullptr;
  const float h = (float)(c->p.dt / c->p.nsub);
  for (int32_t s = 0; s < nsteps; ++s) {
    StepEvents ev;
    int64_t l0 = c->launches;
    if (ps) {
      for (int i = 0; i < 8; ++i) ev.e[i] = prof_event(ps);
      ev.side = 0;
      cudaEventRecord(ev.e[0], c->stream);
    }
    const bool sort_now = c->p.sort_every > 0 && c->step % c->p.sort_every == 0;
    if (c->presorted) {
      // issued during the previous step's field advance
      cudaStreamWaitEvent(c->stream, c->ev_sort, 0);
      c->presorted = 0;
    } else if (sort_now) {
      for (int sp = 0; sp < c->nspecies; ++sp) {
        hv_status st = sort_species(c, sp, c->stream);
        if (st != HV_OK) return st;
      }
      c->since_sort = 0;
    }
    if (ps) {
      cudaEventRecord(ev.e[1], c->stream);
      ev.launches[0] = c->launches - l0;
      l0 = c->launches;
    }
    wait_records(c);
    for (int sp = 0; sp < c->nspecies; ++sp) {
      cudaError_t e = launch_push(c, sp, 0);
      if (e != cudaSuccess) return cuda_fail(e, "push");
    }
    if (c->since_sort >= 0) c->since_sort++;
    if (ps) {
      cudaEventRecord(ev.e[2], c->stream);
      ev.launches[1] = c->launches - l0;
      l0 = c->launches;
    }
    // ions entering through open faces join after the push (Sec. 2.3); the
    // profile counts them with the moment post
    for (int q = 0; q < c->ninject; ++q) {
      cudaError_t e = launch_injection(c, c->inject[q]);
      if (e != cudaSuccess) return cuda_fail(e, "injection");
    }
    // The next step's sort needs only the pushed ions, not the fields: when
    // it is due and runs in this call, issue it now on the side stream so
    // that it overlaps this step's moment post and field advance.  (Its
    // launches count as sort launches; its time shows as the slowdown of the
    // phases it overlaps.)
    if (s + 1 < nsteps && c->p.sort_every > 0 && (c->step + 1) % c->p.sort_every == 0) {
      hv_status st = side_stream(c);
      if (st != HV_OK) return st;
      cudaEventRecord(c->ev_push, c->stream);
      cudaStreamWaitEvent(c->side, c->ev_push, 0);
      if (ps) {
        cudaEventRecord(ev.e[6], c->side);
        ev.side = 1;
      }
      for (int sp = 0; sp < c->nspecies; ++sp) {
        st = sort_species(c, sp, c->side);
        if (st != HV_OK) return st;
      }
      if (ps) cudaEventRecord(ev.e[7], c->side);
      c->since_sort = 0;
      cudaEventRecord(c->ev_sort, c->side);
      c->presorted = 1;
      if (ps) {
        ev.launches[0] += c->launches - l0;
        l0 = c->launches;
      }
    }
    cudaError_t e = launch_moments(c, 0);
    if (e != cudaSuccess) return cuda_fail(e, "moments");
    {
      hv_status rs = clear_records_async(c);
      if (rs != HV_OK) return rs;
    }
    if (ps) {
      cudaEventRecord(ev.e[3], c->stream);
      ev.launches[2] = c->launches - l0;
      l0 = c->launches;
    }
    // the electrostatic model advances no B: only p_e, if it is a field
    const int nsub_run = c->p.ohm_model == 1 && !c->p.pe_eq ? 0 : c->p.nsub;
    for (int k = 0; k < nsub_run; ++k) {
      if (c->p.pe_eq) {
        // B and p_e together (electron energy equation); stage 2 writes in
        // place over its own base cells only
        e = launch_field_stage_pe(c, c->B, c->B, c->Bs, c->pe, c->pe, c->pes, 0.5f * h);
        if (e == cudaSuccess)
          e = launch_field_stage_pe(c, c->Bs, c->B, c->B, c->pes, c->pe, c->pe, h);
      } else if (c->p.ohm_model != 0 || c->g.any_open) {
        // the resistive background: tiled stages
        e = launch_field_stage_tiled(c, c->B, c->B, c->Bs, 0.5f * h);
        if (e == cudaSuccess) e = launch_field_stage_tiled(c, c->Bs, c->B, c->B, h);
      } else if (fused_substeps(c)) {
        // B and B* alternate so that a substep never writes what it reads
        e = launch_substep(c, (k & 1) ? c->Bs : c->B, (k & 1) ? c->B : c->Bs, h);
      } else {
        e = launch_field_stage(c, c->B, c->B, c->Bs, 0.5f * h);
        if (e == cudaSuccess) e = launch_field_stage(c, c->Bs, c->B, c->B, h);
      }
      if (e != cudaSuccess) return cuda_fail(e, "field stage");
    }
    if (!c->p.pe_eq && c->p.ohm_model == 0 && fused_substeps(c) && (c->p.nsub & 1)) {
      // an odd number of fused substeps leaves B^{n+1} in B*: copy it back
      e = cudaMemcpyAsync(c->B, c->Bs, sizeof(float4) * c->g.ncell, cudaMemcpyDeviceToDevice,
                          c->stream);
      if (e != cudaSuccess) return cuda_fail(e, "field copy");
    }
    if (ps) {
      cudaEventRecord(ev.e[4], c->stream);
      ev.launches[3] = c->launches - l0;
      l0 = c->launches;
    }
    e = launch_ohm_final(c, c->mext);
    if (e != cudaSuccess) return cuda_fail(e, "final Ohm");
    if (ps) {
      cudaEventRecord(ev.e[5], c->stream);
      ev.launches[4] = c->launches - l0;
      ps->rec.push_back(ev);
    }
    c->step++;
  }
  return HV_OK;
}

hv_status hv_moments(hv_ctx *c, float *n_out, float *J_out, float *E_out, float *B_out,
                     int on_device) {
  if (!c) return fail(HV_EINVAL, "ctx is NULL");
  if (!c->started) {
    hv_status st = startup(c);
    if (st != HV_OK) return st;
  }
  const Geom &g = c->g;
  const size_t nc = (size_t)g.ncell;
  float *tmp = (float *)dev_alloc(sizeof(float) * 4 * nc, c->stream);
  if (!tmp) return fail(HV_ENOMEM, "hv_moments scratch");
  cudaError_t e = cudaSuccess;
  struct Job {
    float *dst;
    int kind;
  } jobs[4] = {{n_out, 0}, {J_out, 1}, {E_out, 2}, {B_out, 3}};
  for (auto &jb : jobs) {
    if (!jb.dst || e != cudaSuccess) continue;
    int ncomp = jb.kind == 0 ? 1 : 3;
    if (jb.kind == 0) unpack4_kernel<<<eblocks(nc), 256, 0, c->stream>>>(g.ncell, c->mprev, 1, 0, tmp);
    if (jb.kind == 1) unpack4_kernel<<<eblocks(nc), 256, 0, c->stream>>>(g.ncell, c->mprev, 3, 1, tmp);
    if (jb.kind == 2) unpack_E_kernel<<<eblocks(nc), 256, 0, c->stream>>>(g, c->EB, tmp);
    if (jb.kind == 3)
      unpack_B_kernel<<<eblocks(nc), 256, 0, c->stream>>>(g.ncell, c->B, c->B0ext, tmp);
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(jb.dst, tmp, sizeof(float) * ncomp * nc,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
  }
  dev_free(tmp, sizeof(float) * 4 * nc, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_moments");
  return latched(c, nullptr);
}

hv_status hv_electron_pressure(hv_ctx *c, float *pe_out, int on_device) {
  if (!c || !pe_out) return fail(HV_EINVAL, "ctx or pe_out is NULL");
  if (!c->p.pe_eq) return fail(HV_EINVAL, "the context has no electron pressure field (pe_eq = 0)");
  if (!c->started) {
    hv_status st = startup(c);
    if (st != HV_OK) return st;
  }
  cudaError_t e = cudaMemcpyAsync(pe_out, c->pe, sizeof(float) * (size_t)c->g.ncell,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_electron_pressure");
  return latched(c, nullptr);
}

hv_status hv_diag(hv_ctx *c, hv_diag_t *out) {
  if (!c || !out) return fail(HV_EINVAL, "ctx or out is NULL");
  if (!c->started) {
    hv_status st = startup(c);
    if (st != HV_OK) return st;
  }
  cudaError_t e = launch_diag(c);
  double d[8] = {0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d, c->diag_dev, sizeof(double) * 7, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_diag");
  int word = 0;
  hv_status st = latched(c, &word);
  memset(out, 0, sizeof(*out));
  out->step = c->step;
  out->t = c->step * c->p.dt;
  out->W_K = d[0];
  out->P[0] = d[1];
  out->P[1] = d[2];
  out->P[2] = d[3];
  out->charge = d[4];
  out->W_B = d[5];
  out->max_divB = d[6];
  out->err_word = word;
  if (st != HV_OK) return st;
  for (int i = 0; i < 7; ++i)
    if (!std::isfinite(d[i])) return fail(HV_ENAN, "non-finite diagnostic");
  return HV_OK;
}

hv_status hv_diag_async(hv_ctx *c) {
  if (!c) return fail(HV_EINVAL, "ctx is NULL");
  if (c->dq_count == kDiagQueue) return fail(HV_ESTATE, "4 diagnostics pending: wait first");
  if (!c->started) {
    hv_status st = startup(c);
    if (st != HV_OK) return st;
  }
  cudaError_t e = cudaSuccess;
  if (!c->dq_host) {
    e = cudaMallocHost(&c->dq_host, sizeof(DiagSlot) * kDiagQueue);
    for (int i = 0; i < kDiagQueue && e == cudaSuccess; ++i)
      e = cudaEventCreateWithFlags(&c->dq_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "hv_diag_async: host slots");
  }
  DiagSlot &slot = c->dq_host[(c->dq_head + c->dq_count) % kDiagQueue];
  e = launch_diag(c);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(slot.d, c->diag_dev, sizeof(double) * 7, cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&slot.word, c->err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaEventRecord(c->dq_ev[(c->dq_head + c->dq_count) % kDiagQueue], c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_diag_async");
  slot.step = c->step;
  c->dq_count++;
  return HV_OK;
}

hv_status hv_diag_wait(hv_ctx *c, hv_diag_t *out) {
  if (!c || !out) return fail(HV_EINVAL, "ctx or out is NULL");
  if (c->dq_count == 0) return fail(HV_ESTATE, "no diagnostics pending");
  const int i = c->dq_head;
  cudaError_t e = cudaEventSynchronize(c->dq_ev[i]);
  if (e != cudaSuccess) return cuda_fail(e, "hv_diag_wait");
  c->dq_head = (c->dq_head + 1) % kDiagQueue;
  c->dq_count--;
  const DiagSlot &slot = c->dq_host[i];
  memset(out, 0, sizeof(*out));
  out->step = slot.step;
  out->t = slot.step * c->p.dt;
  out->W_K = slot.d[0];
  out->P[0] = slot.d[1];
  out->P[1] = slot.d[2];
  out->P[2] = slot.d[3];
  out->charge = slot.d[4];
  out->W_B = slot.d[5];
  out->max_divB = slot.d[6];
  out->err_word = slot.word;
  const hv_status st = status_of_word(slot.word);
  if (st != HV_OK) return st;
  for (int k = 0; k < 7; ++k)
    if (!std::isfinite(slot.d[k])) return fail(HV_ENAN, "non-finite diagnostic");
  return HV_OK;
}

// hv_get_ions with open faces: the slots in use are read from the device and
// the live ions among them (dead slots skipped) returned in order (host only).
static hv_status get_ions_open(hv_ctx *c, Species &sp, int64_t *n_out, int32_t *cell, float *off3,
                               float *v3, float *w, int on_device) {
  if (on_device) return fail(HV_EINVAL, "with open faces hv_get_ions returns host arrays only");
  int nu = 0;
  cudaError_t e = cudaMemcpyAsync(&nu, sp.n_used, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_get_ions");
  const Soa &s = sp.buf[sp.cur];
  std::vector<int32_t> hc(nu);
  std::vector<float> hf[7];
  const float *src[7] = {s.ox, s.oy, s.oz, s.vx, s.vy, s.vz, s.w};
  if (nu > 0) e = cudaMemcpyAsync(hc.data(), s.cell, 4 * (size_t)nu, cudaMemcpyDeviceToHost, c->stream);
  for (int f = 0; f < 7 && e == cudaSuccess; ++f) {
    hf[f].assign(nu, 0.f);
    if (src[f] && nu > 0)
      e = cudaMemcpyAsync(hf[f].data(), src[f], 4 * (size_t)nu, cudaMemcpyDeviceToHost, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_get_ions");
  int64_t live = 0;
  for (int i = 0; i < nu; ++i) live += hc[i] != kDeadVox;
  if (n_out) *n_out = live;
  int64_t o = 0;
  for (int i = 0; i < nu; ++i) {
    if (hc[i] == kDeadVox) continue;
    if (cell) cell[o] = voxel_to_linear(c->g, hc[i]);
    if (off3) {
      off3[o] = hf[0][i];
      off3[live + o] = hf[1][i];
      off3[2 * live + o] = hf[2][i];
    }
    if (v3) {
      v3[o] = hf[3][i];
      v3[live + o] = hf[4][i];
      v3[2 * live + o] = hf[5][i];
    }
    if (w) w[o] = hf[6][i];
    ++o;
  }
  return latched(c, nullptr);
}

hv_status hv_get_ions(hv_ctx *c, int32_t species, int64_t *n_out, int32_t *cell, float *off3,
                      float *v3, float *w, int on_device) {
  if (!c) return fail(HV_EINVAL, "ctx is NULL");
  if (species < 0 || species >= c->nspecies) return fail(HV_EINVAL, "no such species");
  Species &sp = c->sp[species];
  if (c->g.any_open) return get_ions_open(c, sp, n_out, cell, off3, v3, w, on_device);
  if (n_out) *n_out = sp.n;
  const int64_t n = sp.n;
  const Soa &s = sp.buf[sp.cur];
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void *dst, const void *src) {
    if (dst && e == cudaSuccess && n > 0) e = cudaMemcpyAsync(dst, src, 4 * n, k, c->stream);
  };
  if (cell && n > 0 && e == cudaSuccess) {
    if (on_device) {
      const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8192);
      vox_to_linear_kernel<<<blocks, 256, 0, c->stream>>>(c->g, s.cell, cell, n);
      e = cudaGetLastError();
    } else {
      e = cudaMemcpyAsync(cell, s.cell, 4 * n, k, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      for (int64_t t = 0; t < n && e == cudaSuccess; ++t) cell[t] = voxel_to_linear(c->g, cell[t]);
    }
  }
  if (off3) {
    cp(off3, s.ox);
    if (s.oy) {
      cp(off3 + n, s.oy);
    } else if (n > 0 && e == cudaSuccess) {
      e = on_device ? cudaMemsetAsync(off3 + n, 0, 4 * n, c->stream)
                    : (memset(off3 + n, 0, 4 * n), cudaSuccess);
    }
    cp(off3 + 2 * n, s.oz);
  }
  if (v3) {
    cp(v3, s.vx);
    cp(v3 + n, s.vy);
    cp(v3 + 2 * n, s.vz);
  }
  cp(w, s.w);
  if (e != cudaSuccess) return cuda_fail(e, "hv_get_ions");
  return latched(c, nullptr);
}

hv_status hv_set_filter(hv_ctx *c, const float *params, const float *scale4, double gate_nmin,
                        double gate_rmax) {
  if (!c) return fail(HV_EINVAL, "ctx is NULL");
  if (!params) {
    c->filter_on = 0;
    return HV_OK;
  }
  if (!c->g.dim2) return fail(HV_EINVAL, "the learned filter is built for the x-z layout (ny = 1)");
  if (c->g.any_open) return fail(HV_EINVAL, "the learned filter pads periodically (no open faces)");
  if (!scale4) return fail(HV_EINVAL, "scale4 is NULL");
  for (int i = 0; i < kFilterParams; ++i)
    if (!std::isfinite(params[i])) return fail(HV_EINVAL, "non-finite filter parameter");
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(scale4[i]) || scale4[i] <= 0.f)
      return fail(HV_EINVAL, "filter scales must be finite and > 0");
  if (!std::isfinite(gate_nmin) || !std::isfinite(gate_rmax) || gate_rmax < 0)
    return fail(HV_EINVAL, "gate thresholds must be finite (rmax >= 0)");
  std::vector<__nv_bfloat16> w;
  std::vector<float> bias;
  pack_filter(params, w, bias);
  if (!c->filt.w) {
    c->filt.w = (__nv_bfloat16 *)ctx_alloc(c, sizeof(__nv_bfloat16) * w.size());
    c->filt.bias = (float *)ctx_alloc(c, sizeof(float) * bias.size());
    if (!c->filt.w || !c->filt.bias) return fail(HV_ENOMEM, "filter allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(c->filt.w, w.data(), sizeof(__nv_bfloat16) * w.size(),
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->filt.bias, bias.data(), sizeof(float) * bias.size(),
                        cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_set_filter upload");
  for (int i = 0; i < 4; ++i) c->filt.scale[i] = scale4[i];
  c->filt.nmin = (float)gate_nmin;
  c->filt.rmax = (float)gate_rmax;
  c->filter_on = 1;
  return HV_OK;
}

hv_status hv_filter_moments(hv_ctx *c, const float *m4, float *y4, int on_device) {
  if (!c || !m4 || !y4) return fail(HV_EINVAL, "null argument");
  if (!c->filter_on) return fail(HV_ESTATE, "no filter set");
  const size_t nc = (size_t)c->g.ncell;
  float4 *din = (float4 *)dev_alloc(sizeof(float4) * nc, c->stream);
  float4 *dout = (float4 *)dev_alloc(sizeof(float4) * nc, c->stream);
  if (!din || !dout) {
    dev_free(din, sizeof(float4) * nc, c->stream);
    dev_free(dout, sizeof(float4) * nc, c->stream);
    return fail(HV_ENOMEM, "hv_filter_moments scratch");
  }
  // [4][ncell] component-major in and out
  std::vector<float4> h(nc);
  std::vector<float> hm(4 * nc);
  cudaError_t e = cudaMemcpy(hm.data(), m4, sizeof(float) * 4 * nc,
                             on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
  for (size_t i = 0; i < nc && e == cudaSuccess; ++i)
    h[i] = make_float4(hm[i], hm[nc + i], hm[2 * nc + i], hm[3 * nc + i]);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(din, h.data(), sizeof(float4) * nc, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = launch_filter(c, c->filt, din, dout);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), dout, sizeof(float4) * nc, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dev_free(din, sizeof(float4) * nc, c->stream);
  dev_free(dout, sizeof(float4) * nc, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_filter_moments");
  for (size_t i = 0; i < nc; ++i) {
    hm[i] = h[i].x;
    hm[nc + i] = h[i].y;
    hm[2 * nc + i] = h[i].z;
    hm[3 * nc + i] = h[i].w;
  }
  e = cudaMemcpy(y4, hm.data(), sizeof(float) * 4 * nc,
                 on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost);
  if (e != cudaSuccess) return cuda_fail(e, "hv_filter_moments copy-out");
  return HV_OK;
}

hv_status hv_filter_train_init(hv_ctx *c, const float *params, const float *scale4) {
  if (!c || !params || !scale4) return fail(HV_EINVAL, "null argument");
  hv_status st = hv_set_filter(c, params, scale4, 0.0, 1e30);
  if (st != HV_OK) return st;
  if (!c->tr_P) {
    c->tr_P = (float *)ctx_alloc(c, sizeof(float) * 4 * kFilterParams);
    c->tr_wt = (__nv_bfloat16 *)ctx_alloc(c, sizeof(__nv_bfloat16) * filter_train_weight_count());
    c->tr_loss = (double *)ctx_alloc(c, sizeof(double));
    if (!c->tr_P || !c->tr_wt || !c->tr_loss) return fail(HV_ENOMEM, "training allocation failed");
    c->tr_m1 = c->tr_P + kFilterParams;
    c->tr_m2 = c->tr_m1 + kFilterParams;
    c->tr_grad = c->tr_m2 + kFilterParams;
  }
  std::vector<__nv_bfloat16> wt;
  pack_filter_transposed(params, wt);
  cudaError_t e = cudaMemcpyAsync(c->tr_P, params, sizeof(float) * kFilterParams,
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->tr_m1, 0, sizeof(float) * 3 * kFilterParams, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->tr_wt, wt.data(), sizeof(__nv_bfloat16) * wt.size(),
                        cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_filter_train_init");
  c->tr_step = 0;
  return HV_OK;
}

// gradient (and optionally an Adam step) on nb pairs [nb][4][ncell]
static hv_status filter_train(hv_ctx *c, const float *m, const float *t, int32_t nb, double lr,
                              int update, float *grad_out, double *loss_out, int on_device) {
  if (!c || !m || !t || nb < 1) return fail(HV_EINVAL, "bad training arguments");
  if (!c->tr_P) return fail(HV_ESTATE, "call hv_filter_train_init first");
  const size_t nc = (size_t)c->g.ncell, nfl = 4 * nc * (size_t)nb;
  float *raw = (float *)dev_alloc(sizeof(float) * 2 * nfl, c->stream);
  float4 *il = (float4 *)dev_alloc(sizeof(float4) * 2 * nc * nb, c->stream);
  if (!raw || !il) {
    dev_free(raw, sizeof(float) * 2 * nfl, c->stream);
    dev_free(il, sizeof(float4) * 2 * nc * nb, c->stream);
    return fail(HV_ENOMEM, "training scratch");
  }
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpyAsync(raw, m, sizeof(float) * nfl, k, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(raw + nfl, t, sizeof(float) * nfl, k, c->stream);
  if (e == cudaSuccess) e = launch_interleave4(c, nb, raw, il);
  if (e == cudaSuccess) e = launch_interleave4(c, nb, raw + nfl, il + nc * nb);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->tr_loss, 0, sizeof(double), c->stream);
  if (e == cudaSuccess)
    e = launch_filter_grad(c, c->filt, c->tr_wt, il, il + nc * nb, nb, c->tr_grad, c->tr_loss);
  if (e == cudaSuccess && grad_out)
    e = cudaMemcpyAsync(grad_out, c->tr_grad, sizeof(float) * kFilterParams,
                        cudaMemcpyDeviceToHost, c->stream);
  double loss = 0.0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&loss, c->tr_loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) {
    if (update) {
      c->tr_step++;
      e = launch_adam(c, c->tr_P, c->tr_grad, c->tr_m1, c->tr_m2, c->tr_step, (float)lr, c->filt,
                      c->tr_wt);
    } else {
      e = cudaMemsetAsync(c->tr_grad, 0, sizeof(float) * kFilterParams, c->stream);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dev_free(raw, sizeof(float) * 2 * nfl, c->stream);
  dev_free(il, sizeof(float4) * 2 * nc * nb, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "filter training");
  if (loss_out) *loss_out = loss;
  return HV_OK;
}

hv_status hv_filter_grad(hv_ctx *c, const float *m, const float *t, int32_t nb, float *grad_out,
                         double *loss_out, int on_device) {
  return filter_train(c, m, t, nb, 0.0, 0, grad_out, loss_out, on_device);
}

hv_status hv_filter_train_step(hv_ctx *c, const float *m, const float *t, int32_t nb, double lr,
                               double *loss_out, int on_device) {
  if (!std::isfinite(lr) || lr <= 0) return fail(HV_EINVAL, "lr must be finite and > 0");
  return filter_train(c, m, t, nb, lr, 1, nullptr, loss_out, on_device);
}

hv_status hv_filter_get_params(hv_ctx *c, float *params_out) {
  if (!c || !params_out) return fail(HV_EINVAL, "null argument");
  if (!c->tr_P) return fail(HV_ESTATE, "no training state");
  cudaError_t e = cudaMemcpyAsync(params_out, c->tr_P, sizeof(float) * kFilterParams,
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_filter_get_params");
  return HV_OK;
}

hv_status hv_query(const hv_ctx *c, hv_info_t *out) {
  if (!c || !out) return fail(HV_EINVAL, "ctx or out is NULL");
  memset(out, 0, sizeof(*out));
  out->ncell = c->g.ncell;
  out->tile[0] = c->g.tx;
  out->tile[1] = c->g.ty;
  out->tile[2] = c->g.tz;
  out->ntiles = c->g.ntiles;
  out->nspecies = c->nspecies;
  for (int s = 0; s < c->nspecies; ++s) out->n[s] = c->sp[s].n;
  out->step = c->step;
  return HV_OK;
}

hv_status hv_get_tile_offsets(hv_ctx *c, int32_t species, int32_t *tile_off) {
  if (!c || !tile_off) return fail(HV_EINVAL, "ctx or tile_off is NULL");
  if (species < 0 || species >= c->nspecies) return fail(HV_EINVAL, "no such species");
  cudaError_t e = cudaMemcpyAsync(tile_off, c->sp[species].tile_off,
                                  sizeof(int32_t) * (size_t)(c->g.ntiles + 1),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_get_tile_offsets");
  return latched(c, nullptr);
}

hv_status hv_inject_error(hv_ctx *c, int32_t bits) {
  if (!c) return fail(HV_EINVAL, "ctx is NULL");
  if (bits <= 0 || (bits & ~(kErrCfl | kErrNonFinite | kErrIndex | kErrTimeout | kErrCapacity)))
    return fail(HV_EINVAL, "bits must be a non-empty combination of 1, 2, 4, 8 and 16");
  inject_error_kernel<<<1, 1, 0, c->stream>>>(c->err, bits);
  c->launches++;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "hv_inject_error");
  return HV_OK;
}

hv_status hv_error_status(int32_t err_word) { return status_of_word(err_word); }

hv_status hv_profile(hv_ctx *c, int enable) {
  if (!c) return fail(HV_EINVAL, "ctx is NULL");
  ProfStore *ps = prof_store(c, true);
  cudaStreamSynchronize(c->stream);
  prof_recycle(ps);
  memset(&c->prof, 0, sizeof(c->prof));
  c->prof_on = enable ? 1 : 0;
  c->prof.launches = 0;
  c->launches = 0;
  return HV_OK;
}

hv_status hv_profile_read(hv_ctx *c, hv_prof_t *out) {
  if (!c || !out) return fail(HV_EINVAL, "ctx or out is NULL");
  ProfStore *ps = prof_store(c, true);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_profile_read");
  for (auto &r : ps->rec) {
    float ms[5] = {0, 0, 0, 0, 0};
    for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&ms[i], r.e[i], r.e[i + 1]);
    if (r.side) {
      float side_ms = 0.f;
      cudaEventElapsedTime(&side_ms, r.e[6], r.e[7]);
      ms[0] += side_ms;
    }
    c->prof.ms_sort += ms[0];
    c->prof.ms_push += ms[1];
    c->prof.ms_moments += ms[2];
    c->prof.ms_field += ms[3];
    c->prof.ms_ohm += ms[4];
    c->prof.n_sort += r.launches[0];
    c->prof.n_push += r.launches[1];
    c->prof.n_moments += r.launches[2];
    c->prof.n_field += r.launches[3];
    c->prof.n_ohm += r.launches[4];
    c->prof.steps += 1;
  }
  prof_recycle(ps);
  c->prof.launches = c->launches;
  *out = c->prof;
  return HV_OK;
}

void hv_destroy(hv_ctx *c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaEventDestroy(c->ev_push);
    cudaEventDestroy(c->ev_sort);
    cudaEventDestroy(c->ev_fold);
    cudaEventDestroy(c->ev_rec[0]);
    cudaEventDestroy(c->ev_rec[1]);
    cudaStreamDestroy(c->side);
  }
  prof_destroy(c);
  if (c->dq_host) {
    for (int i = 0; i < kDiagQueue; ++i)
      if (c->dq_ev[i]) cudaEventDestroy(c->dq_ev[i]);
    cudaFreeHost(c->dq_host);
  }
  for (int s = 0; s < c->nspecies; ++s) {
    for (int b = 0; b < 2; ++b) dev_free(c->sp[s].base[b], c->sp[s].bytes[b], c->stream);
    dev_free(std::min(c->sp[s].tile_off, c->sp[s].tile_off_next),
             sizeof(int) * 2 * (c->g.ntiles + 1), c->stream);
  }
  sort_release(c);
  for (int i = 0; i < c->nallocs; ++i) dev_free(c->allocs[i], c->alloc_bytes[i], c->stream);
  cudaStreamSynchronize(c->stream);
  delete c;
}

hv_status hv_sort_keys(const int32_t *keys, int64_t n, int32_t nkeys, int32_t *perm,
                       int32_t *counts, void *cuda_stream) {
  return sort_keys(keys, n, nkeys, perm, counts, (cudaStream_t)cuda_stream, nullptr);
}

}  // extern "C"
