// Sorting (a device of the GPU layout: it keeps a warp's particles in one or
// two cells so that gathers hit shared memory and deposits aggregate; the
// method's result changes only through FP32 summation order).
//
// The step sorts each species by supercell key with a stable counting sort
// (sort_species): ions of one key keep their order, so the permutation is
// that of a plain stable counting sort of the keys.  It has a general path
// and a windowed path for ions that moved at most a few cells since the last
// sort (described before sort_species below).  The general path, and the
// stable key sort of the ABI (hv_sort_keys), is a least-significant-digit
// radix sort on (key, index) pairs with 8-bit digits, ceil(log2(nkeys)/8)
// passes.  Each pass is reduce-then-scan, so no kernel waits on another
// block:
//   upsweep   per 4096-key tile digit counts -> table[digit][tile]
//   scan      exclusive scan of the table in digit-major order
//   downsweep stable per-tile ranks (warp match + per-warp counters) and
//             scatter to table offset + rank.
// The particles are then gathered by the permutation, or (after an earlier
// sort) the last pass writes every original index's sorted position instead
// and a final pass reads the particle arrays in order and stores every
// particle at its position.
#include <algorithm>

#include "hv_internal.cuh"

namespace hv {

struct SortScratch {
  int32_t *k[2], *v[2];
  int32_t *table, *bsum;
  int64_t cap_n, cap_table, cap_bsum;
  void *base;
  size_t bytes;
};

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // 4096
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kScanChunk = 4096;

// radix passes: a lane loads all of its 16 items before it counts or ranks
// any (off: item by item)
#ifndef HV_RADIX_PREFETCH
#define HV_RADIX_PREFETCH 1
#endif
// downsweep: a tile's items are ordered by digit in shared memory before
// they are stored, so that the stores of one digit are contiguous (off:
// every item stored from its lane)
#ifndef HV_RADIX_STAGE
#define HV_RADIX_STAGE 1
#endif
// general sort of ions sorted before: place them at their sorted positions
// (off: gather them by the permutation, as the first sort does)
#ifndef HV_GENERAL_PLACE
#define HV_GENERAL_PLACE 1
#endif

// Items of a tile are split into one contiguous run of 512 per warp; round r
// of warp w covers tile items w*512 + r*32 + lane, so lane order within a
// round and round order within a warp follow input order.
__device__ __forceinline__ int64_t item_index(int64_t tile0, int warp, int r, int lane) {
  return tile0 + warp * (32 * kItems) + r * 32 + lane;
}

__global__ void __launch_bounds__(kThreads) upsweep_kernel(const int32_t *keys, int64_t n,
                                                            int shift, int64_t ntiles,
                                                            int32_t *table) {
  __shared__ int hist[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  hist[threadIdx.x] = 0;
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * kTile;
#if HV_RADIX_PREFETCH
  // every key of the lane loaded before the first count
  int key[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t idx = item_index(tile0, warp, r, lane);
    key[r] = idx < n ? keys[idx] : 0;
  }
#pragma unroll
#endif
  for (int r = 0; r < kItems; ++r) {
    const int64_t idx = item_index(tile0, warp, r, lane);
    const bool valid = idx < n;
    const unsigned act = __ballot_sync(kFull, valid);
    if (!valid) continue;
#if HV_RADIX_PREFETCH
    const int d = (int)(((uint32_t)key[r] >> shift) & 255u);
#else
    const int d = (int)(((uint32_t)keys[idx] >> shift) & 255u);
#endif
    const unsigned peers = __match_any_sync(act, d);
    if (lane == __ffs(peers) - 1) atomicAdd(&hist[d], __popc(peers));
  }
  __syncthreads();
  table[(int64_t)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

// Exclusive scan of a large int32 array in three steps: chunk sums, scan of
// the sums in one block, chunk-local scans plus the chunk offset.
__global__ void __launch_bounds__(kThreads) chunk_sum_kernel(const int32_t *a, int64_t len,
                                                              int32_t *bsum) {
  __shared__ int s[kThreads];
  const int64_t c0 = (int64_t)blockIdx.x * kScanChunk;
  int t = 0;
  for (int i = threadIdx.x; i < kScanChunk; i += kThreads) {
    const int64_t idx = c0 + i;
    if (idx < len) t += a[idx];
  }
  s[threadIdx.x] = t;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}

// block-wide exclusive scan of one value per thread; returns the total
__device__ int block_exclusive_scan(int x, int *s_warp, int &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < kWarps ? s_warp[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += y;
    }
    if (lane < kWarps) s_warp[lane] = wi - w;
    if (lane == kWarps - 1) s_warp[kWarps] = wi;
  }
  __syncthreads();
  total = s_warp[kWarps];
  const int r = s_warp[warp] + incl - x;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kThreads) scan_bsum_kernel(int32_t *bsum, int64_t nb) {
  __shared__ int s_warp[kWarps + 1];
  int carry = 0;
  for (int64_t base = 0; base < nb; base += kThreads) {
    const int64_t idx = base + threadIdx.x;
    const int x = idx < nb ? bsum[idx] : 0;
    int total;
    const int ex = block_exclusive_scan(x, s_warp, total);
    if (idx < nb) bsum[idx] = carry + ex;
    carry += total;
  }
}

__global__ void __launch_bounds__(kThreads) chunk_scan_kernel(int32_t *a, int64_t len,
                                                               const int32_t *bsum) {
  __shared__ int s_warp[kWarps + 1];
  const int64_t c0 = (int64_t)blockIdx.x * kScanChunk;
  int carry = bsum[blockIdx.x];
  constexpr int per = kScanChunk / kThreads;  // 16 consecutive values per thread
  int v[per];
  int t = 0;
  for (int i = 0; i < per; ++i) {
    const int64_t idx = c0 + (int64_t)threadIdx.x * per + i;
    v[i] = idx < len ? a[idx] : 0;
    t += v[i];
  }
  int total;
  int ex = block_exclusive_scan(t, s_warp, total) + carry;
  for (int i = 0; i < per; ++i) {
    const int64_t idx = c0 + (int64_t)threadIdx.x * per + i;
    if (idx < len) a[idx] = ex;
    ex += v[i];
  }
}

// vals_out receives the values in sorted order, or with `inverse` the
// sorted position of every value at index value (the inverse permutation
// when the values are the original indices).
__global__ void __launch_bounds__(kThreads) downsweep_kernel(const int32_t *keys_in,
                                                              const int32_t *vals_in, int64_t n,
                                                              int shift, int64_t ntiles,
                                                              const int32_t *table,
                                                              int32_t *keys_out,
                                                              int32_t *vals_out, bool inverse) {
  __shared__ int wcount[kWarps][256];
  __shared__ int gbase[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int w = 0; w < kWarps; ++w) wcount[w][threadIdx.x] = 0;
  gbase[threadIdx.x] = table[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * kTile;
  int key[kItems], val[kItems], rank[kItems];
#if HV_RADIX_PREFETCH
  // every key and value of the lane loaded before the first rank
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t idx = item_index(tile0, warp, r, lane);
    const bool valid = idx < n;
    key[r] = valid ? keys_in[idx] : 0;
    val[r] = valid ? (vals_in ? vals_in[idx] : (int)idx) : 0;
  }
#endif
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t idx = item_index(tile0, warp, r, lane);
    const bool valid = idx < n;
#if !HV_RADIX_PREFETCH
    key[r] = valid ? keys_in[idx] : 0;
    val[r] = valid ? (vals_in ? vals_in[idx] : (int)idx) : 0;
#endif
    rank[r] = -1;
    const unsigned act = __ballot_sync(kFull, valid);
    if (valid) {
      const int d = (int)(((uint32_t)key[r] >> shift) & 255u);
      const unsigned peers = __match_any_sync(act, d);
      const int before = wcount[warp][d];
      rank[r] = before + __popc(peers & ((1u << lane) - 1u));
      __syncwarp(act);
      if (lane == __ffs(peers) - 1) wcount[warp][d] = before + __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  // exclusive scan over warps for each digit (thread = digit)
  int total = 0;
  for (int w = 0; w < kWarps; ++w) {
    const int t = wcount[w][threadIdx.x];
    wcount[w][threadIdx.x] = total;
    total += t;
  }
#if HV_RADIX_STAGE
  __shared__ int skey[kTile], sval[kTile];
  __shared__ int dstart[256], wsum[kWarps];
  // the tile's first position of every digit: exclusive scan of the digit
  // totals
  int incl = total;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += wsum[w];
  dstart[threadIdx.x] = before + incl - total;
  __syncthreads();
  // every item to its position in the tile ordered by digit (stable: warp,
  // round, lane order), then stored from there in that order
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    if (rank[r] < 0) continue;
    const int d = (int)(((uint32_t)key[r] >> shift) & 255u);
    const int loc = dstart[d] + wcount[warp][d] + rank[r];
    skey[loc] = key[r];
    sval[loc] = val[r];
  }
  __syncthreads();
  const int nv = (int)min((int64_t)kTile, n - tile0);
  for (int j = threadIdx.x; j < nv; j += kThreads) {
    const int k = skey[j];
    const int d = (int)(((uint32_t)k >> shift) & 255u);
    const int64_t dst = (int64_t)gbase[d] + (j - dstart[d]);
    keys_out[dst] = k;
    if (inverse) vals_out[sval[j]] = (int32_t)dst;
    else vals_out[dst] = sval[j];
  }
#else
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    if (rank[r] < 0) continue;
    const int d = (int)(((uint32_t)key[r] >> shift) & 255u);
    const int64_t dst = (int64_t)gbase[d] + wcount[warp][d] + rank[r];
    keys_out[dst] = key[r];
    if (inverse) vals_out[val[r]] = (int32_t)dst;
    else vals_out[dst] = val[r];
  }
#endif
}

// Count keys (warp-aggregated atomics) and flag out-of-range keys.  The loop
// advances whole warps together so that every lane of a warp takes part in
// the ballot and match of each round.
__global__ void count_kernel(const int32_t *keys, int64_t n, int32_t nkeys, int32_t *counts,
                             int *bad) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
       base += stride) {
    const int64_t i = base + lane;
    const int k = i < n ? keys[i] : 0;
    const bool inrange = i < n && k >= 0 && k < nkeys;
    if (i < n && !inrange) atomicOr(bad, 1);
    const unsigned act = __ballot_sync(kFull, inrange);
    if (!inrange || !counts) continue;
    const unsigned peers = __match_any_sync(act, k);
    if (lane == __ffs(peers) - 1) atomicAdd(&counts[k], __popc(peers));
  }
}

int key_bits(int64_t nkeys) {
  int b = 1;
  while (b < 31 && ((int64_t)1 << b) < nkeys) ++b;
  return b;
}

int64_t table_len(int64_t n) { return 256 * ((n + kTile - 1) / kTile); }

int64_t bsum_len(int64_t len) { return (len + kScanChunk - 1) / kScanChunk; }

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Size (or resize) the scratch for n keys.  Returns false on allocation
// failure.
bool scratch_reserve(SortScratch *&s, int64_t n, cudaStream_t st) {
  const int64_t tl = table_len(std::max<int64_t>(n, 1));
  const int64_t bl = bsum_len(tl);
  if (s && s->cap_n >= n && s->cap_table >= tl && s->cap_bsum >= bl) return true;
  if (s) {
    dev_free(s->base, s->bytes, st);
  } else {
    s = new SortScratch();
  }
  const int64_t nn = std::max<int64_t>(n, 1);
  const size_t kv = align256(sizeof(int32_t) * nn);
  const size_t bytes = 4 * kv + align256(sizeof(int32_t) * tl) + align256(sizeof(int32_t) * bl);
  char *p = (char *)dev_alloc(bytes, st);
  if (!p) {
    delete s;
    s = nullptr;
    return false;
  }
  s->base = p;
  s->bytes = bytes;
  s->k[0] = (int32_t *)p;
  s->k[1] = (int32_t *)(p + kv);
  s->v[0] = (int32_t *)(p + 2 * kv);
  s->v[1] = (int32_t *)(p + 3 * kv);
  s->table = (int32_t *)(p + 4 * kv);
  s->bsum = (int32_t *)(p + 4 * kv + align256(sizeof(int32_t) * tl));
  s->cap_n = nn;
  s->cap_table = tl;
  s->cap_bsum = bl;
  return true;
}

// Radix passes over keys[n]; returns the buffers holding the permutation
// (with `inverse`, the sorted position of every input index instead) and
// the sorted keys.
cudaError_t radix_perm(const int32_t *keys, int64_t n, int64_t nkeys, SortScratch *s,
                       cudaStream_t st, int32_t **perm_out, int64_t *launches,
                       int32_t **keys_out = nullptr, bool inverse = false) {
  const int bits = key_bits(nkeys);
  const int passes = (bits + 7) / 8;
  const int64_t ntiles = (n + kTile - 1) / kTile;
  const int64_t tl = 256 * ntiles;
  const int64_t nb = bsum_len(tl);
  const int32_t *kin = keys;
  const int32_t *vin = nullptr;
  int out = 0;
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    upsweep_kernel<<<(unsigned)ntiles, kThreads, 0, st>>>(kin, n, shift, ntiles, s->table);
    chunk_sum_kernel<<<(unsigned)nb, kThreads, 0, st>>>(s->table, tl, s->bsum);
    scan_bsum_kernel<<<1, kThreads, 0, st>>>(s->bsum, nb);
    chunk_scan_kernel<<<(unsigned)nb, kThreads, 0, st>>>(s->table, tl, s->bsum);
    downsweep_kernel<<<(unsigned)ntiles, kThreads, 0, st>>>(kin, vin, n, shift, ntiles, s->table,
                                                             s->k[out], s->v[out],
                                                             inverse && p == passes - 1);
    *launches += 5;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kin = s->k[out];
    vin = s->v[out];
    out ^= 1;
  }
  *perm_out = const_cast<int32_t *>(vin);
  if (keys_out) *keys_out = const_cast<int32_t *>(kin);
  return cudaSuccess;
}

// ----------------------------------------------------------------------------
// The step's sort: a stable counting sort of the ions by supercell key (tile,
// then cell in the tile); ions with equal keys keep the order they had.  An
// ion's key cell is its cell moved by at most one cell along an axis on
// which its offset plus its velocity times kSortHorizon * sort_every * dt /
// Delta leaves [-1, 1): the cell it is predicted to reach 0.6875 sort
// intervals later (pred_shift; none with open faces).  Ions leave their
// sorted cells in both directions between two sorts instead of in one,
// which halves the deposit runs the push has to break.  Two paths give the
// same permutation:
//
// General path (the first sort after loading, long sort intervals): the keys
// go through the stable radix passes above, the ions are gathered by the
// permutation (the first sort) or stored at their sorted positions (later
// sorts), and the tile ranges are found by binary search in the sorted keys.
//
// Windowed path: between two sorts an ion moves at most one cell per axis
// per step (a larger move is a CFL error and the ion is held), and a key
// cell is at most one cell from the ion's cell at either sort, so when at
// most H - 2 steps have passed (H with no prediction), every ion of tile t's
// last range [tile_off[t], tile_off[t+1]) has its key cell in t's window:
// the tile grown by H cells on each side, periodically.  A cell's position
// in that window is its slot.
//   rank:    one block per tile walks the tile's range in order, each warp
//            a contiguous part with warp-private slot counters; a first walk
//            counts, an exclusive scan over the warps turns the counts into
//            starting ranks, a second walk gives every ion its rank among
//            the earlier ions of the range in the same slot;
//   prefix:  per key, the tiles whose windows hold its cell, in tile order:
//            each (tile, slot) count becomes the number of ions of that key
//            in earlier tiles' ranges, and their sum is the key's count;
//   scan:    counts -> offsets (in place), tile ranges from the offsets;
//   base:    per (tile, slot) the key's offset plus that prefix;
//   scatter: one ion per thread moves to base[tile][slot] + rank.
// ----------------------------------------------------------------------------
template <int DIM>
struct SortWin {
  static constexpr int TX = DIM == 2 ? kTile2X : kTile3;
  static constexpr int TY = DIM == 2 ? 1 : kTile3;
  static constexpr int TZ = DIM == 2 ? kTile2Z : kTile3;
  static constexpr int H = DIM == 2 ? 10 : 4;  // window halo in cells
  static constexpr int WX = TX + 2 * H, WY = DIM == 2 ? 1 : TY + 2 * H, WZ = TZ + 2 * H;
  static constexpr int NS = WX * WY * WZ;     // slots per window
  static constexpr int WARPS = DIM == 2 ? 8 : 4;
  static constexpr size_t rank_smem = sizeof(int32_t) * WARPS * NS;
  static_assert(NS <= 65536, "slots are cached as 16-bit values");
};

// ions per lane whose loads the rank kernel's walks issue together
#ifndef HV_SORT_UNROLL
#define HV_SORT_UNROLL 4
#endif
constexpr int kSortUnroll = HV_SORT_UNROLL;

// v mod n in [0, n) (v is almost always already in range)
__device__ __forceinline__ int wrap0(int v, int n) {
  if (v >= 0 && v < n) return v;
  v %= n;
  return v < 0 ? v + n : v;
}

// Interior cell of a voxel index; false for a voxel that is not interior.
__device__ __forceinline__ bool vox_cell(const Geom &g, int vox, int &i, int &j, int &k) {
  if (vox < g.vlo || vox >= g.vhi) return false;
  const uint32_t v = (uint32_t)vox;
  const uint32_t q = fdiv(v, g.div_px);
  i = (int)(v - q * (uint32_t)g.px) - kGhost;
  if (g.dim2) {
    j = 0;
    k = (int)q - kGhost;
  } else {
    const int kp = (int)fdiv(q, g.div_py);
    j = (int)q - kp * g.py - kGhost;
    k = kp - kGhost;
  }
  return (unsigned)i < (unsigned)g.nx && (unsigned)j < (unsigned)g.ny &&
         (unsigned)k < (unsigned)g.nz;
}

// Origin cell of tile t.
template <int DIM>
__device__ __forceinline__ void tile_origin(const Geom &g, int t, int &x0, int &y0, int &z0) {
  using SW = SortWin<DIM>;
  x0 = (t % g.ntx) * SW::TX;
  y0 = ((t / g.ntx) % g.nty) * SW::TY;
  z0 = (t / (g.ntx * g.nty)) * SW::TZ;
}

// Slot of cell (i, j, k) in the window of the tile with origin (x0, y0, z0),
// or -1 outside it.  The periodic offset is taken in [0, n) per axis, so
// every cell has one slot even where the window is wider than the grid.
template <int DIM>
__device__ __forceinline__ int win_slot(const Geom &g, int x0, int y0, int z0, int i, int j,
                                        int k) {
  using SW = SortWin<DIM>;
  const int sx = wrap0(i - x0 + SW::H, g.nx);
  const int sz = wrap0(k - z0 + SW::H, g.nz);
  const int sy = DIM == 2 ? 0 : wrap0(j - y0 + SW::H, g.ny);
  if (sx >= SW::WX || sy >= SW::WY || sz >= SW::WZ) return -1;
  return sx + SW::WX * (sy + SW::WY * sz);
}

// Slot of an ion's key cell (its cell moved by the predicted shift) in tile
// t's window; an ion that is not in the window (only a corrupt cell index
// can do that) takes slot 0 and raises the index error.
template <int DIM>
__device__ __forceinline__ int ion_slot(const Geom &g, int x0, int y0, int z0, int vox, int sx,
                                        int sy, int sz, bool &bad) {
  int i, j, k;
  int s = -1;
  if (vox_cell(g, vox, i, j, k))
    s = win_slot<DIM>(g, x0, y0, z0, wrap1(i + sx, g.nx), wrap1(j + sy, g.ny),
                      wrap1(k + sz, g.nz));
  if (s < 0) {
    bad = true;
    s = 0;
  }
  return s;
}

template <int DIM>
__global__ void __launch_bounds__(SortWin<DIM>::WARPS * 32)
    wsort_rank_kernel(Geom g, Soa ions, const int *tile_off, int32_t *wcnt, int32_t *rank,
                      uint16_t *slot_cache, int *err) {
  using SW = SortWin<DIM>;
  extern __shared__ int32_t cw[];  // [WARPS][NS] warp-private slot counters
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = blockIdx.x;
  int x0, y0, z0;
  tile_origin<DIM>(g, t, x0, y0, z0);
  for (int s = threadIdx.x; s < SW::WARPS * SW::NS; s += blockDim.x) cw[s] = 0;
  __syncthreads();
  const int a = tile_off[t], b = tile_off[t + 1];
  const int64_t len = b - a;
  const int wa = a + (int)(len * warp / SW::WARPS), wb = a + (int)(len * (warp + 1) / SW::WARPS);
  int32_t *mine = cw + warp * SW::NS;
  const unsigned lt = (1u << lane) - 1u;
  bool bad = false;
  for (int walk = 0; walk < 2; ++walk) {
    for (int base = wa; base < wb; base += 32 * kSortUnroll) {
      int sl[kSortUnroll];
      if (walk == 0) {
        // the first walk computes the slots and keeps them for the second
        int v[kSortUnroll], sx[kSortUnroll], sy[kSortUnroll], sz[kSortUnroll];
#pragma unroll
        for (int u = 0; u < kSortUnroll; ++u) {
          const int idx = base + 32 * u + lane;
          v[u] = 0;
          sx[u] = sy[u] = sz[u] = 0;
          if (idx < wb) {
            v[u] = ions.cell[idx];
            sx[u] = pred_shift(ions.ox[idx], ions.vx[idx], g.pcx);
            if (DIM == 3) sy[u] = pred_shift(ions.oy[idx], ions.vy[idx], g.pcy);
            sz[u] = pred_shift(ions.oz[idx], ions.vz[idx], g.pcz);
          }
        }
#pragma unroll
        for (int u = 0; u < kSortUnroll; ++u) {
          const int idx = base + 32 * u + lane;
          sl[u] = idx < wb ? ion_slot<DIM>(g, x0, y0, z0, v[u], sx[u], sy[u], sz[u], bad) : 0;
          if (idx < wb) slot_cache[idx] = (uint16_t)sl[u];
        }
      } else {
#pragma unroll
        for (int u = 0; u < kSortUnroll; ++u) {
          const int idx = base + 32 * u + lane;
          sl[u] = idx < wb ? (int)slot_cache[idx] : 0;
        }
      }
#pragma unroll
      for (int u = 0; u < kSortUnroll; ++u) {
        const int idx = base + 32 * u + lane;
        const unsigned act = __ballot_sync(kFull, idx < wb);
        if (idx < wb) {
          const unsigned peers = __match_any_sync(act, sl[u]);
          const int before = mine[sl[u]];
          __syncwarp(act);
          if (lane == __ffs(peers) - 1) mine[sl[u]] = before + __popc(peers);
          if (walk == 1) rank[idx] = before + __popc(peers & lt);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (walk == 0) {
      // per slot: the warps' counts -> their starting ranks; the tile's total
      for (int s = threadIdx.x; s < SW::NS; s += blockDim.x) {
        int run = 0;
#pragma unroll
        for (int w = 0; w < SW::WARPS; ++w) {
          const int c = cw[w * SW::NS + s];
          cw[w * SW::NS + s] = run;
          run += c;
        }
        wcnt[(size_t)t * SW::NS + s] = run;
      }
      __syncthreads();
    }
  }
  if (bad) atomicOr(err, kErrIndex);
}

// Distinct tile coordinates T-1, T, T+1 (periodic) on an axis of n tiles.
__device__ __forceinline__ int tile_neighbours(int T, int n, int *out) {
  int c = 0;
  const int cand[3] = {T == 0 ? n - 1 : T - 1, T, T == n - 1 ? 0 : T + 1};
  for (int q = 0; q < 3; ++q) {
    bool dup = false;
    for (int r = 0; r < c; ++r) dup = dup || out[r] == cand[q];
    if (!dup) out[c++] = cand[q];
  }
  return c;
}

template <int DIM>
__global__ void __launch_bounds__(256) wsort_prefix_kernel(Geom g, int32_t *wcnt, int32_t *cnt) {
  using SW = SortWin<DIM>;
  const int nkeys = g.ntiles << g.tlog;
  for (int key = blockIdx.x * blockDim.x + threadIdx.x; key < nkeys;
       key += gridDim.x * blockDim.x) {
    const int T = key >> g.tlog, l = key & ((1 << g.tlog) - 1);
    const int Tx = T % g.ntx, Ty = (T / g.ntx) % g.nty, Tz = T / (g.ntx * g.nty);
    const int i = Tx * SW::TX + l % SW::TX;
    const int j = Ty * SW::TY + (l / SW::TX) % SW::TY;
    const int k = Tz * SW::TZ + l / (SW::TX * SW::TY);
    if (i >= g.nx || j >= g.ny || k >= g.nz) {  // a cell of a ragged tile that does not exist
      cnt[key] = 0;
      continue;
    }
    int cx[3], cy[3], cz[3];
    const int nxc = tile_neighbours(Tx, g.ntx, cx);
    const int nyc = DIM == 2 ? 1 : tile_neighbours(Ty, g.nty, cy);
    if (DIM == 2) cy[0] = 0;
    const int nzc = tile_neighbours(Tz, g.ntz, cz);
    int cand[27];
    int nc = 0;
    for (int c3 = 0; c3 < nzc; ++c3)
      for (int c2 = 0; c2 < nyc; ++c2)
        for (int c1 = 0; c1 < nxc; ++c1) {
          // insertion into ascending order: ranges lie in tile order
          const int v = cx[c1] + g.ntx * (cy[c2] + g.nty * cz[c3]);
          int p = nc++;
          while (p > 0 && cand[p - 1] > v) {
            cand[p] = cand[p - 1];
            --p;
          }
          cand[p] = v;
        }
    // the windows that hold the cell, their counts all loaded before any
    // prefix is stored (the loads overlap instead of waiting on each store)
    int at[27], cn[27];
    int m = 0;
    for (int q = 0; q < nc; ++q) {
      int x0, y0, z0;
      tile_origin<DIM>(g, cand[q], x0, y0, z0);
      const int s = win_slot<DIM>(g, x0, y0, z0, i, j, k);
      if (s < 0) continue;
      at[m++] = cand[q] * SW::NS + s;
    }
    for (int q = 0; q < m; ++q) cn[q] = wcnt[at[q]];
    int run = 0;
    for (int q = 0; q < m; ++q) {
      wcnt[at[q]] = run;
      run += cn[q];
    }
    cnt[key] = run;
  }
}

// First destination of every (tile, slot): the key's offset plus the count
// of its ions in earlier tiles' ranges (in place over the prefixes).
template <int DIM>
__global__ void __launch_bounds__(256) wsort_base_kernel(Geom g, int32_t *wpre,
                                                         const int32_t *off) {
  using SW = SortWin<DIM>;
  const int64_t total = (int64_t)g.ntiles * SW::NS;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / SW::NS), s = (int)(e - (int64_t)t * SW::NS);
    int x0, y0, z0;
    tile_origin<DIM>(g, t, x0, y0, z0);
    const int sx = s % SW::WX, sy = (s / SW::WX) % SW::WY, sz = s / (SW::WX * SW::WY);
    const int i = wrap0(x0 - SW::H + sx, g.nx);
    const int j = DIM == 2 ? 0 : wrap0(y0 - SW::H + sy, g.ny);
    const int k = wrap0(z0 - SW::H + sz, g.nz);
    wpre[e] += off[supercell_key(g, i, j, k)];
  }
}

// The scatter over the whole array: a warp takes 32 * kScatItems
// consecutive ions, lane l the ions warp_base + 32 m + l.  Every ion's fields
// are loaded first, so that the loads overlap one another and the search
// for the tile range holding the warp's first ion (binary search in
// tile_off by lane 0); the lanes then step forward across range ends, and
// an ion goes to wbase[tile][slot] + rank.  (One ion per lane: 771 us at
// 1024x512 against 823 us with the loads after the search; 2 and 4 ions
// per lane took 930 and 1065 us.)
#ifndef HV_WSCATTER_ITEMS
#define HV_WSCATTER_ITEMS 1
#endif
constexpr int kScatItems = HV_WSCATTER_ITEMS;

template <int DIM>
__global__ void __launch_bounds__(256) wsort_scatter_flat_kernel(Geom g, Soa in, Soa out, int64_t n,
                                                                 const int *tile_off,
                                                                 const int32_t *wbase,
                                                                 const int32_t *rank) {
  using SW = SortWin<DIM>;
  const int lane = threadIdx.x & 31;
  const int64_t wbase0 =
      ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 * kScatItems);
  if (wbase0 >= n) return;
  int c[kScatItems], r[kScatItems];
  float x[kScatItems], y[kScatItems], z[kScatItems], vx[kScatItems], vy[kScatItems],
      vz[kScatItems], w[kScatItems];
#pragma unroll
  for (int m = 0; m < kScatItems; ++m) {
    const int64_t i = wbase0 + 32 * m + lane;
    c[m] = 0;
    r[m] = 0;
    x[m] = y[m] = z[m] = vx[m] = vy[m] = vz[m] = w[m] = 0.f;
    if (i < n) {
      c[m] = in.cell[i];
      r[m] = rank[i];
      x[m] = in.ox[i];
      if (DIM == 3) y[m] = in.oy[i];
      z[m] = in.oz[i];
      vx[m] = in.vx[i];
      vy[m] = in.vy[i];
      vz[m] = in.vz[i];
      w[m] = in.w[i];
    }
  }
  int t = 0;
  if (lane == 0) {
    int lo = 0, hi = g.ntiles;  // last tile whose range starts at or before wbase0
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if ((int64_t)__ldg(tile_off + mid) <= wbase0) lo = mid;
      else hi = mid;
    }
    t = lo;
  }
  t = __shfl_sync(kFull, t, 0);
#pragma unroll
  for (int m = 0; m < kScatItems; ++m) {
    const int64_t i = wbase0 + 32 * m + lane;
    if (i >= n) break;
    while (t + 1 < g.ntiles && (int64_t)__ldg(tile_off + t + 1) <= i) ++t;
    int x0, y0, z0;
    tile_origin<DIM>(g, t, x0, y0, z0);
    bool bad = false;
    const int sx = pred_shift(x[m], vx[m], g.pcx),
              sy = DIM == 3 ? pred_shift(y[m], vy[m], g.pcy) : 0,
              sz = pred_shift(z[m], vz[m], g.pcz);
    const int d = __ldg(wbase + (size_t)t * SW::NS +
                        ion_slot<DIM>(g, x0, y0, z0, c[m], sx, sy, sz, bad)) +
                  r[m];
    out.cell[d] = c[m];
    out.ox[d] = x[m];
    if (DIM == 3) out.oy[d] = y[m];
    out.oz[d] = z[m];
    out.vx[d] = vx[m];
    out.vy[d] = vy[m];
    out.vz[d] = vz[m];
    out.w[d] = w[m];
  }
}

// General path: keys, gather by permutation, tile ranges from sorted keys.
// (a dead slot, open faces, takes the key after the last one: behind every
// live ion)
__global__ void ion_keys_kernel(Geom g, Soa ions, int64_t n, int32_t *keys) {
  const int dead_key = g.ntiles << g.tlog;
  const bool has_y = ions.oy != nullptr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int v = ions.cell[i];
    const int sx = pred_shift(ions.ox[i], ions.vx[i], g.pcx);
    const int sy = has_y ? pred_shift(ions.oy[i], ions.vy[i], g.pcy) : 0;
    const int sz = pred_shift(ions.oz[i], ions.vz[i], g.pcz);
    keys[i] = v == kDeadVox ? dead_key : ion_key(g, v, sx, sy, sz);
  }
}

// slots in use after a sort with open faces: the live ions (the dead sorted
// behind them)
__global__ void live_count_kernel(const int *tile_off, int ntiles, int *n_used) {
  *n_used = tile_off[ntiles];
}

// Ion perm[i] to position i (stores in order, reads scattered).
__global__ void gather_kernel(Soa in, Soa out, const int32_t *perm, int64_t n) {
  const bool has_y = in.oy != nullptr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = perm[i];
    out.cell[i] = in.cell[s];
    out.ox[i] = in.ox[s];
    if (has_y) out.oy[i] = in.oy[s];
    out.oz[i] = in.oz[s];
    out.vx[i] = in.vx[s];
    out.vy[i] = in.vy[s];
    out.vz[i] = in.vz[s];
    out.w[i] = in.w[s];
  }
}

// Ion i (read in order) to its sorted position dst[i]: the reads are
// coalesced and only the stores scatter, which do not hold a thread up.
__global__ void __launch_bounds__(256) place_kernel(Soa in, Soa out, const int32_t *dst, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool has_y = in.oy != nullptr;
  const int64_t d = dst[i];
  const int c = in.cell[i];
  const float ox = in.ox[i], oy = has_y ? in.oy[i] : 0.f, oz = in.oz[i];
  const float vx = in.vx[i], vy = in.vy[i], vz = in.vz[i], w = in.w[i];
  out.cell[d] = c;
  out.ox[d] = ox;
  if (has_y) out.oy[d] = oy;
  out.oz[d] = oz;
  out.vx[d] = vx;
  out.vy[d] = vy;
  out.vz[d] = vz;
  out.w[d] = w;
}

// tile_off[t] = first index whose sorted key is >= t << tlog (binary search)
__global__ void tile_bounds_kernel(const int32_t *skeys, int64_t n, int tlog, int ntiles,
                                   int *tile_off) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles; t += gridDim.x * blockDim.x) {
    const int64_t target = (int64_t)t << tlog;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if ((int64_t)skeys[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    tile_off[t] = (int)lo;
  }
}

// Tile ranges from the scanned key counts: tile t starts at its first key.
__global__ void tile_starts_kernel(const int32_t *off, int tlog, int ntiles, int64_t n, int *tile_off) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles; t += gridDim.x * blockDim.x)
    tile_off[t] = t == ntiles ? (int)n : off[(int64_t)t << tlog];
}

__global__ void tile_even_kernel(int64_t n, int ntiles, int *off) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles; t += gridDim.x * blockDim.x)
    off[t] = (int)(n * t / ntiles);
}

}  // namespace

namespace {

// Per-species scratch of the windowed path: key counts (scanned in place
// into offsets), the scan's chunk sums, every ion's rank, and the per-tile
// window counts; allocated at the species' first windowed sort.
template <int DIM>
hv_status window_reserve(hv_ctx *c, Species &sp, int32_t **cnt, int32_t **bsum, int32_t **rank,
                         uint16_t **slots) {
  const Geom &g = c->g;
  const int64_t nkeys = (int64_t)g.ntiles << g.tlog;
  const int64_t nb = bsum_len(nkeys);
  const size_t kb = align256(sizeof(int32_t) * nkeys), bb = align256(sizeof(int32_t) * nb);
  const size_t rb = align256(sizeof(int32_t) * std::max<int64_t>(sp.n, 1));
  if (!sp.bucket) {
    sp.bucket_bytes = kb + bb + rb + align256(sizeof(uint16_t) * std::max<int64_t>(sp.n, 1));
    sp.bucket = (int32_t *)dev_alloc(sp.bucket_bytes, c->stream);
    if (!sp.bucket) return fail(HV_ENOMEM, "sort scratch allocation failed");
  }
  if (!sp.wcnt) {
    sp.wcnt_bytes = sizeof(int32_t) * (size_t)g.ntiles * SortWin<DIM>::NS;
    sp.wcnt = (int32_t *)dev_alloc(sp.wcnt_bytes, c->stream);
    if (!sp.wcnt) return fail(HV_ENOMEM, "sort window allocation failed");
  }
  *cnt = sp.bucket;
  *bsum = (int32_t *)((char *)sp.bucket + kb);
  *rank = (int32_t *)((char *)sp.bucket + kb + bb);
  *slots = (uint16_t *)((char *)sp.bucket + kb + bb + rb);
  return HV_OK;
}

template <int DIM>
hv_status sort_windowed(hv_ctx *c, Species &sp, cudaStream_t st) {
  using SW = SortWin<DIM>;
  const Geom &g = c->g;
  int32_t *cnt, *bsum, *rank;
  uint16_t *slots;
  hv_status hs = window_reserve<DIM>(c, sp, &cnt, &bsum, &rank, &slots);
  if (hs != HV_OK) return hs;
  static std::atomic<uint64_t> attr_rank{0};
  cudaError_t e = set_smem_once(wsort_rank_kernel<DIM>, SW::rank_smem, attr_rank);
  if (e != cudaSuccess) return cuda_fail(e, "sort kernel attributes");
  const int64_t nkeys = (int64_t)g.ntiles << g.tlog;
  const int64_t nb = bsum_len(nkeys);
  const Soa &src = sp.buf[sp.cur];
  wsort_rank_kernel<DIM><<<g.ntiles, SW::WARPS * 32, SW::rank_smem, st>>>(
      g, src, sp.tile_off, sp.wcnt, rank, slots, c->err);
  wsort_prefix_kernel<DIM><<<(unsigned)((nkeys + 255) / 256), 256, 0, st>>>(g, sp.wcnt, cnt);
  chunk_sum_kernel<<<(unsigned)nb, kThreads, 0, st>>>(cnt, nkeys, bsum);
  scan_bsum_kernel<<<1, kThreads, 0, st>>>(bsum, nb);
  chunk_scan_kernel<<<(unsigned)nb, kThreads, 0, st>>>(cnt, nkeys, bsum);
  tile_starts_kernel<<<(g.ntiles + 256) / 256, 256, 0, st>>>(cnt, g.tlog, g.ntiles, sp.n,
                                                             sp.tile_off_next);
  const int64_t tot = (int64_t)g.ntiles * SW::NS;
  wsort_base_kernel<DIM><<<(unsigned)std::min<int64_t>((tot + 255) / 256, 8 * 2048), 256, 0, st>>>(
      g, sp.wcnt, cnt);
  wsort_scatter_flat_kernel<DIM>
      <<<(unsigned)((sp.n + 256 * kScatItems - 1) / (256 * kScatItems)), 256, 0, st>>>(
          g, src, sp.buf[sp.cur ^ 1], sp.n, sp.tile_off, sp.wcnt, rank);
  c->launches += 8;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "windowed sort");
  return HV_OK;
}

hv_status sort_general(hv_ctx *c, Species &sp, cudaStream_t st) {
  const Geom &g = c->g;
  if (!scratch_reserve(c->sort, sp.n, st)) return fail(HV_ENOMEM, "sort scratch allocation failed");
  SortScratch *s = c->sort;
  const int64_t nkeys = (int64_t)g.ntiles << g.tlog;
  const Soa &src = sp.buf[sp.cur];
  const int eb = (int)std::min<int64_t>((sp.n + 255) / 256, 8 * 2048);
  // the keys live in v[1]: the first radix pass reads them and writes
  // k[0], v[0]; later passes overwrite them only after that
  ion_keys_kernel<<<eb, 256, 0, st>>>(g, src, sp.n, s->v[1]);
  // ions in the order they were loaded in are gathered (scattered reads,
  // stores in order); ions sorted before move little, and placing them
  // (reads in order, stores mostly in runs) is faster
  const bool place = HV_GENERAL_PLACE && c->since_sort >= 0;
  int32_t *idx = nullptr, *skeys = nullptr;
  int64_t launches = 1;
  cudaError_t e = radix_perm(s->v[1], sp.n, nkeys + (g.any_open ? 1 : 0), s, st, &idx,
                             &launches, &skeys, /*inverse=*/place);
  if (e == cudaSuccess) {
    if (place)
      place_kernel<<<(unsigned)((sp.n + 255) / 256), 256, 0, st>>>(src, sp.buf[sp.cur ^ 1], idx,
                                                                   sp.n);
    else
      gather_kernel<<<(unsigned)((sp.n + 255) / 256), 256, 0, st>>>(src, sp.buf[sp.cur ^ 1], idx,
                                                                    sp.n);
    tile_bounds_kernel<<<(g.ntiles + 256) / 256, 256, 0, st>>>(skeys, sp.n, g.tlog, g.ntiles,
                                                              sp.tile_off_next);
    launches += 2;
    if (g.any_open) {
      live_count_kernel<<<1, 1, 0, st>>>(sp.tile_off_next, g.ntiles, sp.n_used);
      launches++;
    }
    e = cudaGetLastError();
  }
  c->launches += launches;
  if (e != cudaSuccess) return cuda_fail(e, "general sort");
  return HV_OK;
}

}  // namespace

int sort_window(const hv_ctx *c) { return c->g.dim2 ? SortWin<2>::H : SortWin<3>::H; }

hv_status sort_species(hv_ctx *c, int sidx, cudaStream_t stream) {
  Species &sp = c->sp[sidx];
  if (sp.n == 0) return HV_OK;
  // (open faces: dead slots must be sorted out, which the general path does;
  // a predicted key cell is at most one cell from the ion's cell, at this
  // sort and at the last one)
  const bool pred = c->g.pcx != 0.f || c->g.pcy != 0.f || c->g.pcz != 0.f;
  const bool windowed = !c->g.any_open && c->since_sort >= 0 &&
                        c->since_sort + (pred ? 2 : 0) <= sort_window(c);
  hv_status st;
  if (windowed)
    st = c->g.dim2 ? sort_windowed<2>(c, sp, stream) : sort_windowed<3>(c, sp, stream);
  else
    st = sort_general(c, sp, stream);
  if (st != HV_OK) return st;
  sp.cur ^= 1;
  std::swap(sp.tile_off, sp.tile_off_next);
  return HV_OK;
}

cudaError_t tile_ranges_even(hv_ctx *c, int s) {
  Species &sp = c->sp[s];
  tile_even_kernel<<<(c->g.ntiles + 256) / 256, 256, 0, c->stream>>>(sp.n, c->g.ntiles,
                                                                       sp.tile_off);
  c->launches++;
  return cudaGetLastError();
}

void sort_release(hv_ctx *c) {
  if (c->sort) {
    dev_free(c->sort->base, c->sort->bytes, c->stream);
    delete c->sort;
    c->sort = nullptr;
  }
  for (int s = 0; s < kMaxSpecies; ++s) {
    Species &sp = c->sp[s];
    if (sp.bucket) dev_free(sp.bucket, sp.bucket_bytes, c->stream);
    if (sp.wcnt) dev_free(sp.wcnt, sp.wcnt_bytes, c->stream);
    sp.bucket = nullptr;
    sp.wcnt = nullptr;
  }
}

hv_status sort_keys(const int32_t *keys, int64_t n, int32_t nkeys, int32_t *perm, int32_t *counts,
                    cudaStream_t st, int64_t *launches) {
  if (n < 0 || nkeys < 1) return fail(HV_EINVAL, "hv_sort_keys: n < 0 or nkeys < 1");
  if (n > 0 && (!keys || !perm)) return fail(HV_EINVAL, "hv_sort_keys: null pointer");
  if (n >= ((int64_t)1 << 31)) return fail(HV_EINVAL, "hv_sort_keys: n must be < 2^31");
  int64_t dummy = 0;
  if (!launches) launches = &dummy;
  int *bad = (int *)dev_alloc(sizeof(int), st);
  if (!bad) return fail(HV_ENOMEM, "hv_sort_keys: allocation failed");
  cudaMemsetAsync(bad, 0, sizeof(int), st);
  hv_status rc = HV_OK;
  SortScratch *s = nullptr;
  if (counts) cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)nkeys, st);
  if (n > 0) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8 * 1024);
    count_kernel<<<blocks, 256, 0, st>>>(keys, n, nkeys, counts, bad);
    ++*launches;
  }
  if (n > 0) {
    if (!scratch_reserve(s, n, st)) {
      rc = fail(HV_ENOMEM, "hv_sort_keys: scratch allocation failed");
    } else {
      int32_t *p = nullptr;
      cudaError_t e = radix_perm(keys, n, nkeys, s, st, &p, launches);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(perm, p, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) rc = cuda_fail(e, "hv_sort_keys");
    }
  }
  int hbad = 0;
  cudaError_t e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess && rc == HV_OK) rc = cuda_fail(e, "hv_sort_keys sync");
  if (s) {
    dev_free(s->base, s->bytes, st);
    delete s;
  }
  dev_free(bad, sizeof(int), st);
  if (rc == HV_OK && hbad) rc = fail(HV_EINVAL, "hv_sort_keys: key out of range");
  return rc;
}

}  // namespace hv

// ----------------------------------------------------------------------------
// Key sort without any allocation: the same passes as hv_sort_keys, with their
// scratch in one static device array that every GPU loading the library
// holds until the process exits.
// ----------------------------------------------------------------------------
namespace hv {
namespace {

constexpr int64_t kNoAllocMaxKeys = int64_t(1) << 20;  // 1,048,576 keys
constexpr int64_t kNoAllocTable = 256 * ((kNoAllocMaxKeys + kTile - 1) / kTile);
constexpr int64_t kNoAllocBsum = (kNoAllocTable + kScanChunk - 1) / kScanChunk;
// words: keys x2, values x2, digit table, chunk sums, error flag (+ padding)
constexpr int64_t kNoAllocWords = 4 * kNoAllocMaxKeys + kNoAllocTable + kNoAllocBsum + 64;

// About 16.3 MB of device memory per GPU.
static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocWords];

// Device address of the static scratch in the current context, looked up on
// every call: a cached address would outlive a cudaDeviceReset, which
// rebuilds the primary context and its module globals.
hv_status noalloc_base(int32_t **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess)
    return cuda_fail(e, "hv_sort_keys_noalloc: cudaGetSymbolAddress of the static scratch");
  *out = static_cast<int32_t *>(p);
  return HV_OK;
}

}  // namespace
}  // namespace hv

extern "C" hv_status hv_sort_keys_noalloc(const int32_t *keys, int64_t n, int32_t nkeys,
                                          int32_t *perm, int32_t *counts, void *cuda_stream) {
  using namespace hv;
  if (n < 0 || nkeys < 1) return fail(HV_EINVAL, "hv_sort_keys_noalloc: n < 0 or nkeys < 1");
  if (n > kNoAllocMaxKeys)
    return fail(HV_EINVAL,
                "hv_sort_keys_noalloc: n exceeds the 1048576-key limit of its static scratch");
  if (n > 0 && (!keys || !perm)) return fail(HV_EINVAL, "hv_sort_keys_noalloc: null pointer");
  int32_t *base = nullptr;
  hv_status st = noalloc_base(&base);
  if (st != HV_OK) return st;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  SortScratch s;
  s.k[0] = base;
  s.k[1] = base + kNoAllocMaxKeys;
  s.v[0] = base + 2 * kNoAllocMaxKeys;
  s.v[1] = base + 3 * kNoAllocMaxKeys;
  s.table = base + 4 * kNoAllocMaxKeys;
  s.bsum = s.table + kNoAllocTable;
  int *bad = reinterpret_cast<int *>(s.bsum + kNoAllocBsum);
  s.cap_n = kNoAllocMaxKeys;
  s.cap_table = kNoAllocTable;
  s.cap_bsum = kNoAllocBsum;
  s.base = base;
  s.bytes = 0;
  // the flag and the counts must start at zero; every other word is written
  // by the passes before it is read
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), stream);
  if (e == cudaSuccess && counts)
    e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)nkeys, stream);
  int64_t launches = 0;
  if (e == cudaSuccess && n > 0) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8 * 1024);
    count_kernel<<<blocks, 256, 0, stream>>>(keys, n, nkeys, counts, bad);
    e = cudaGetLastError();
    int32_t *p = nullptr;
    if (e == cudaSuccess) e = radix_perm(keys, n, nkeys, &s, stream, &p, &launches);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(perm, p, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, stream);
  }
  int hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "hv_sort_keys_noalloc");
  if (hbad) return fail(HV_EINVAL, "hv_sort_keys_noalloc: key out of range");
  return HV_OK;
}
