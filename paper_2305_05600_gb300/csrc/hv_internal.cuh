// Internal declarations shared by the libhv translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/hv.h"

namespace hv {

constexpr int kMaxSpecies = 8;

// Device error bits latched by kernels (atomicOr into the error word).
constexpr int kErrCfl = 1;     // a particle moved more than one cell in a step
constexpr int kErrNonFinite = 2;
constexpr int kErrIndex = 4;    // a corrupt cell index was skipped

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

// Geometry of the ghost-padded gather/deposit grids: one ghost layer on each
// side of every axis; padded index p = (i+1) + PX*((j+1) + PY*(k+1)).
// In the 2D (x-z) layout the y axis is not padded: p = (i+1) + PX*(k+1).
struct Geom {
  int nx, ny, nz;
  int px, py, pz;       // padded extents (2D: py = 1)
  int sx, sy, sz;       // padded strides (x: 1)
  int ncell;            // interior cells
  int npad;             // padded cells
  int dim2;             // 1: x-z plane layout (ny == 1)
  FastDiv div_nx, div_ny;
};

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
  Soa buf[2];
  int cur;              // index of the live buffer set
  void *base[2];        // allocation bases
  size_t bytes[2];
};

struct PushConsts {
  float qmdt2;          // (q/m) dt / 2
  float cx, cy, cz;     // dt / Delta per axis (0 for single-cell axes)
  float qvc;            // q / V_c
  float mass;           // m
};

struct SortScratch;

}  // namespace hv

struct hv_ctx {
  hv_params p;
  hv::Geom g;
  cudaStream_t stream;
  int device;
  double vc;
  // grids (device)
  float4 *EB;           // padded [npad][2]: {Ex,Ey,Ez,Bx},{By,Bz,0,0}
  float4 *acc;          // padded [npad] deposit accumulator {n,Jx,Jy,Jz}
  float4 *B, *Bs;       // interior [ncell] {Bx,By,Bz,0}
  float4 *mhalf, *mext, *mprev, *mtmp;  // interior moments {n,Jx,Jy,Jz}
  double *pushpart;     // [kMaxSpecies][push_blocks][4]
  double *gridpart;     // [grid_blocks][4]
  double *diag_dev;     // [8]
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

// kernels launchers (return cudaGetLastError of the launch)
cudaError_t launch_push(hv_ctx *c, int species, int mode);
cudaError_t launch_moments(hv_ctx *c, int init);
cudaError_t launch_field_stage(hv_ctx *c, const float4 *Bin, const float4 *Bbase, float4 *Bout,
                               float coef);
cudaError_t launch_ohm_final(hv_ctx *c, const float4 *mom);
cudaError_t launch_diag(hv_ctx *c);
int push_grid_blocks(int device);
int grid_reduce_blocks(int device);

// sort: sorts species `s` of the context by cell (stable), swapping buffers
hv_status sort_species(hv_ctx *c, int s);
void sort_release(hv_ctx *c);
// standalone key sort into perm with scratch from the allocation hook
hv_status sort_keys(const int32_t *keys, int64_t n, int32_t nkeys, int32_t *perm,
                    int32_t *counts, cudaStream_t stream, int64_t *launches);

}  // namespace hv
