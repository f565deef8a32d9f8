// Injection of ions through open faces (Sec. 2.3): after the push of a step,
// every face cell of an open face with an injection set draws new ions from
// the flux of a drifting Maxwellian (density n, flow u, temperature T, ion
// weight w; after Daughton et al. 2006, as the paper cites):
//  * the expected count per face cell and step, N = Gamma A dt / w with the
//    one-sided flux Gamma = n [vt/sqrt(2 pi) exp(-U^2/2vt^2)
//    + U/2 (1 + erf(U/(sqrt2 vt)))] (U the inward flow, vt = sqrt(T/m)), is
//    computed on the host as a 40.24 fixed-point number and rounded
//    stochastically in integer arithmetic: count = (N + (r >> 8)) >> 24;
//  * ion k of a cell takes its inward speed from the flux-weighted
//    distribution (40 bisections of its distribution function), its
//    tangential velocity from the Maxwellian (Box-Muller), its tangential
//    position uniformly in the face cell, and its depth v_n dt u from a
//    uniform entry time in the step; an ion that would lie beyond the grid
//    keeps a dead slot;
//  * the random words come from Philox4x32-10 (Salmon, Moraes, Dror and
//    Shaw, SC 2011) at counter (step, face cell, k or 0xffffffff for the
//    count, species << 8 | face << 4 | call), keyed by the run's seed.
// Counts are scanned so that ions are appended in face-cell order after the
// slots in use; they deposit from the next step on.
#include <cmath>

#include "hv_internal.cuh"

namespace hv {
namespace {

struct InjArgs {
  Geom g;
  Soa s;
  int *n_used;
  int64_t cap;
  int *err;
  int *counts;           // [ncells + 1] counts, then exclusive offsets + total
  int ncells;
  uint32_t step, key0, key1, tag;
  unsigned long long nfix;
  int ax, t1, t2, low;   // face axis, tangential axes (ascending), low face
  float vt, a, sgn, dt;  // thermal speed, inward flow / vt, inward sign, step
  float u[3];
  float w, delta_n;      // ion weight, cell size along the face normal
  int n[3];
};

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1, uint32_t *out) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// a 32-bit word as a uniform in [0, 1) with 24 bits (exact in float)
__device__ __forceinline__ float u24(uint32_t x) { return (float)(x >> 8) * (1.f / 16777216.f); }

// inward speed in units of vt with flux-weighted distribution function u:
// g(t) = exp(-a^2/2) - exp(-(t-a)^2/2) + a sqrt(pi/2) [erf((t-a)/sqrt2) +
// erf(a/sqrt2)], bisected 40 times on [0, max(a, 0) + 12]
__device__ float flux_speed(float a, float u) {
  const float s2 = 1.41421356237309505f, sp2 = 1.25331413731550025f;  // sqrt 2, sqrt(pi/2)
  const float e0 = expf(-0.5f * a * a), ea = erff(a / s2);
  const float ginf = e0 + a * sp2 * (1.f + ea);
  float lo = 0.f, hi = fmaxf(a, 0.f) + 12.f;
  for (int it = 0; it < 40; ++it) {
    const float mid = 0.5f * (lo + hi);
    const float gm = e0 - expf(-0.5f * (mid - a) * (mid - a)) + a * sp2 * (erff((mid - a) / s2) + ea);
    if (gm < u * ginf) lo = mid;
    else hi = mid;
  }
  return 0.5f * (lo + hi);
}

__global__ void inject_count_kernel(InjArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.ncells) return;
  uint32_t r[4];
  philox4x32_10(a.step, (uint32_t)c, 0xffffffffu, a.tag, a.key0, a.key1, r);
  a.counts[c] = (int)((a.nfix + (unsigned long long)(r[0] >> 8)) >> 24);
}

// exclusive scan of the counts in one block; counts[ncells] = total
__global__ void __launch_bounds__(1024) inject_scan_kernel(int *counts, int ncells) {
  __shared__ int s[1024];
  int carry = 0;
  for (int base = 0; base < ncells; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < ncells ? counts[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < ncells) counts[i] = carry + s[threadIdx.x] - v;
    carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[ncells] = carry;
}

__global__ void inject_fill_kernel(InjArgs a, const int *raw) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.ncells) return;
  uint32_t r[4];
  philox4x32_10(a.step, (uint32_t)c, 0xffffffffu, a.tag, a.key0, a.key1, r);
  const int count = (int)((a.nfix + (unsigned long long)(r[0] >> 8)) >> 24);
  const int i1 = c % a.n[a.t1], i2 = c / a.n[a.t1];
  const int64_t base = (int64_t)*a.n_used + a.counts[c];
  const bool has_y = a.s.oy != nullptr;
  for (int k = 0; k < count; ++k) {
    const int64_t slot = base + k;
    if (slot >= a.cap) {
      atomicOr(a.err, kErrCapacity);
      return;
    }
    uint32_t ra[4], rb[4];
    philox4x32_10(a.step, (uint32_t)c, (uint32_t)k, a.tag, a.key0, a.key1, ra);
    philox4x32_10(a.step, (uint32_t)c, (uint32_t)k, a.tag | 1u, a.key0, a.key1, rb);
    const float vn = a.vt > 0.f ? a.vt * flux_speed(a.a, u24(ra[0])) : a.sgn * a.u[a.ax];
    const float rr = sqrtf(-2.f * logf(1.f - u24(ra[1])));
    float sn, cs;
    sincospif(2.f * u24(ra[2]), &sn, &cs);
    const float depth = vn * a.dt * u24(rb[2]) / a.delta_n;  // cells from the face
    const float xr = a.low ? depth : (float)a.n[a.ax] - depth;
    const float fl = floorf(xr);
    int ci[3];
    float o[3], v[3];
    ci[a.ax] = (int)fl;
    o[a.ax] = 2.f * (xr - fl) - 1.f;
    v[a.ax] = a.sgn * vn;
    ci[a.t1] = i1;
    ci[a.t2] = i2;
    o[a.t1] = a.n[a.t1] > 1 ? 2.f * u24(rb[0]) - 1.f : 0.f;
    o[a.t2] = a.n[a.t2] > 1 ? 2.f * u24(rb[1]) - 1.f : 0.f;
    v[a.t1] = a.u[a.t1] + a.vt * rr * cs;
    v[a.t2] = a.u[a.t2] + a.vt * rr * sn;
    const bool inside = fl >= 0.f && fl < (float)a.n[a.ax] && o[a.ax] < 1.f;
    a.s.cell[slot] = inside ? voxel_of(a.g, ci[0], ci[1], ci[2]) : kDeadVox;
    a.s.ox[slot] = o[0];
    if (has_y) a.s.oy[slot] = o[1];
    a.s.oz[slot] = o[2];
    a.s.vx[slot] = v[0];
    a.s.vy[slot] = v[1];
    a.s.vz[slot] = v[2];
    a.s.w[slot] = a.w;
  }
  (void)raw;
}

__global__ void inject_commit_kernel(int *n_used, const int *counts, int ncells, int64_t cap) {
  const int64_t t = (int64_t)*n_used + counts[ncells];
  *n_used = (int)(t < cap ? t : cap);
}

}  // namespace

cudaError_t launch_injection(hv_ctx *c, const InjectFace &f) {
  Species &sp = c->sp[f.species];
  const Geom &g = c->g;
  InjArgs a;
  a.g = g;
  a.s = sp.buf[sp.cur];
  a.n_used = sp.n_used;
  a.cap = sp.n;
  a.err = c->err;
  a.ax = f.face / 2;
  a.low = f.face % 2 == 0;
  a.t1 = a.ax == 0 ? 1 : 0;
  a.t2 = a.ax == 2 ? 1 : 2;
  a.n[0] = g.nx;
  a.n[1] = g.ny;
  a.n[2] = g.nz;
  a.ncells = a.n[a.t1] * a.n[a.t2];
  a.counts = c->inj_scratch;
  const double d[3] = {c->p.dx, c->p.dy, c->p.dz};
  const double m = sp.m;
  const double vt = std::sqrt(f.T / m), sgn = a.low ? 1.0 : -1.0, U = sgn * f.u[a.ax];
  double flux;
  if (vt > 0.0)
    flux = f.n * (vt / std::sqrt(2.0 * 3.14159265358979323846) * std::exp(-U * U / (2.0 * vt * vt)) +
                  0.5 * U * (1.0 + std::erf(U / (std::sqrt(2.0) * vt))));
  else
    flux = f.n * (U > 0.0 ? U : 0.0);
  const double area = d[(a.ax + 1) % 3] * d[(a.ax + 2) % 3];
  const double N = flux * area * c->p.dt / f.w;
  a.nfix = (unsigned long long)std::floor(N * 16777216.0 + 0.5);
  a.step = (uint32_t)c->step;
  a.key0 = (uint32_t)c->p.seed;
  a.key1 = (uint32_t)(c->p.seed >> 32);
  a.tag = ((uint32_t)f.species << 8) | ((uint32_t)f.face << 4);
  a.vt = (float)vt;
  a.a = vt > 0.0 ? (float)(U / vt) : 0.f;
  a.sgn = (float)sgn;
  a.dt = (float)c->p.dt;
  for (int q = 0; q < 3; ++q) a.u[q] = (float)f.u[q];
  a.w = (float)f.w;
  a.delta_n = (float)d[a.ax];
  const int blocks = (a.ncells + 255) / 256;
  inject_count_kernel<<<blocks, 256, 0, c->stream>>>(a);
  inject_scan_kernel<<<1, 1024, 0, c->stream>>>(a.counts, a.ncells);
  inject_fill_kernel<<<blocks, 256, 0, c->stream>>>(a, nullptr);
  inject_commit_kernel<<<1, 1, 0, c->stream>>>(sp.n_used, a.counts, a.ncells, a.cap);
  c->launches += 4;
  return cudaGetLastError();
}

}  // namespace hv
