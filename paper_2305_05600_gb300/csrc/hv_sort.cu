// Sorting (a device of the GPU layout: it keeps a warp's particles in one or
// two cells so that gathers hit shared memory and deposits aggregate; the
// method's result changes only through FP32 summation order).
//
// The step sorts each species by supercell key with one counting-sort pass
// (sort_species).  The stable key sort of the ABI (hv_sort_keys) is a
// least-significant-digit radix sort on (key, index) pairs with 8-bit
// digits, ceil(log2(nkeys)/8) passes.  Each pass is reduce-then-scan, so no
// kernel waits on another block:
//   upsweep   per 4096-key tile digit counts -> table[digit][tile]
//   scan      exclusive scan of the table in digit-major order
//   downsweep stable per-tile ranks (warp match + per-warp counters) and
//             scatter to table offset + rank.
// A final gather applies the permutation to the particle arrays.
#include <algorithm>
#include <mutex>

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
  for (int r = 0; r < kItems; ++r) {
    const int64_t idx = item_index(tile0, warp, r, lane);
    const bool valid = idx < n;
    const unsigned act = __ballot_sync(kFull, valid);
    if (!valid) continue;
    const int d = (int)(((uint32_t)keys[idx] >> shift) & 255u);
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

__global__ void __launch_bounds__(kThreads) downsweep_kernel(const int32_t *keys_in,
                                                              const int32_t *vals_in, int64_t n,
                                                              int shift, int64_t ntiles,
                                                              const int32_t *table,
                                                              int32_t *keys_out,
                                                              int32_t *vals_out) {
  __shared__ int wcount[kWarps][256];
  __shared__ int gbase[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int w = 0; w < kWarps; ++w) wcount[w][threadIdx.x] = 0;
  gbase[threadIdx.x] = table[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  __syncthreads();
  const int64_t tile0 = (int64_t)blockIdx.x * kTile;
  int key[kItems], val[kItems], rank[kItems];
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t idx = item_index(tile0, warp, r, lane);
    const bool valid = idx < n;
    key[r] = valid ? keys_in[idx] : 0;
    val[r] = valid ? (vals_in ? vals_in[idx] : (int)idx) : 0;
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
  // exclusive scan over warps for each digit
  {
    int run = 0;
    for (int w = 0; w < kWarps; ++w) {
      const int t = wcount[w][threadIdx.x];
      wcount[w][threadIdx.x] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    if (rank[r] < 0) continue;
    const int d = (int)(((uint32_t)key[r] >> shift) & 255u);
    const int64_t dst = (int64_t)gbase[d] + wcount[warp][d] + rank[r];
    keys_out[dst] = key[r];
    vals_out[dst] = val[r];
  }
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

// Radix passes over keys[n]; returns the buffers holding the permutation and
// the sorted keys.
cudaError_t radix_perm(const int32_t *keys, int64_t n, int64_t nkeys, SortScratch *s,
                       cudaStream_t st, int32_t **perm_out, int64_t *launches,
                       int32_t **keys_out = nullptr) {
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
                                                             s->k[out], s->v[out]);
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

// The step's sort: a counting sort of the ions by supercell key.  Counts
// and ranks (warp-aggregated atomics), an exclusive scan of the counts,
// then every ion is copied once to its key's offset plus its rank.  Ions
// of one key keep no particular order among themselves (the atomics'
// order); the deposit sums them in any order.
// Each warp takes kUnroll consecutive chunks of 32 ions per iteration and
// issues all their loads (and, in the count, all their atomics) before it
// needs a result, so memory latencies overlap.
constexpr int kUnroll = 4;

// Key counts with warp-aggregated atomics; the value an atomic returns
// gives every ion its rank among the ions of its key, which the scatter
// uses to place it without atomics of its own.
__global__ void bucket_count_kernel(Geom g, const int32_t *vox, int64_t n, int32_t *cnt,
                                    int32_t *rank) {
  const int lane = threadIdx.x & 31;
  const int64_t wstride = (int64_t)gridDim.x * blockDim.x * kUnroll;
  for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31)) * kUnroll;
       base < n; base += wstride) {
    int v[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = base + 32 * u + lane;
      v[u] = i < n ? vox[i] : 0;
    }
    int r[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = base + 32 * u + lane;
      const unsigned act = __ballot_sync(kFull, i < n);
      if (i >= n) continue;
      const int key = ion_key(g, v[u]);
      const unsigned peers = __match_any_sync(act, key);
      const int leader = __ffs(peers) - 1;
      int first = 0;
      if (lane == leader) first = atomicAdd(&cnt[key], __popc(peers));
      first = __shfl_sync(act, first, leader);
      r[u] = first + __popc(peers & ((1u << lane) - 1u));
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t i = base + 32 * u + lane;
      if (i < n) rank[i] = r[u];
    }
  }
}

// Copy every ion to off[key] + rank.  (Issuing several ions' loads per
// thread measured no faster: at a sort every few steps the drifted ions
// make short store segments, and those, not load latency, set the pace.)
__global__ void bucket_scatter_kernel(Geom g, Soa in, Soa out, int64_t n, const int32_t *off,
                                      const int32_t *rank) {
  const bool has_y = in.oy != nullptr;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
    const int c = in.cell[i];
    const float x = in.ox[i];
    const float y = has_y ? in.oy[i] : 0.f;
    const float z = in.oz[i];
    const float vx = in.vx[i], vy = in.vy[i], vz = in.vz[i], w = in.w[i];
    const int d = __ldg(off + ion_key(g, c)) + rank[i];
    out.cell[d] = c;
    out.ox[d] = x;
    if (has_y) out.oy[d] = y;
    out.oz[d] = z;
    out.vx[d] = vx;
    out.vy[d] = vy;
    out.vz[d] = vz;
    out.w[d] = w;
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

// Per-species key counts, scan sums and ion ranks, allocated at the first
// sort.
hv_status bucket_reserve(hv_ctx *c, Species &sp, int32_t **cnt, int32_t **bsum,
                         int32_t **rank) {
  const Geom &g = c->g;
  const int64_t nkeys = (int64_t)g.ntiles << g.tlog;
  const int64_t nb = bsum_len(nkeys);
  const size_t kb = align256(sizeof(int32_t) * nkeys), bb = align256(sizeof(int32_t) * nb);
  if (!sp.bucket) {
    sp.bucket_bytes = kb + bb + align256(sizeof(int32_t) * std::max<int64_t>(sp.n, 1));
    sp.bucket = (int32_t *)dev_alloc(sp.bucket_bytes, c->stream);
    if (!sp.bucket) return fail(HV_ENOMEM, "sort scratch allocation failed");
  }
  *cnt = sp.bucket;
  *bsum = (int32_t *)((char *)sp.bucket + kb);
  *rank = (int32_t *)((char *)sp.bucket + kb + bb);
  return HV_OK;
}

// Counts of the live buffer's keys and every ion's rank in its key, the
// counts scanned in place into offsets, and the tile starts taken from them
// into tile_off.
cudaError_t key_offsets(hv_ctx *c, Species &sp, int32_t *cnt, int32_t *bsum, int32_t *rank,
                        int *tile_off, cudaStream_t st) {
  const Geom &g = c->g;
  const int64_t nkeys = (int64_t)g.ntiles << g.tlog;
  const int64_t nb = bsum_len(nkeys);
  const int blocks = (int)std::max<int64_t>((sp.n + 1023) / 1024, 1);
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nkeys, st);
  if (e != cudaSuccess) return e;
  bucket_count_kernel<<<blocks, 256, 0, st>>>(g, sp.buf[sp.cur].cell, sp.n, cnt, rank);
  chunk_sum_kernel<<<(unsigned)nb, kThreads, 0, st>>>(cnt, nkeys, bsum);
  scan_bsum_kernel<<<1, kThreads, 0, st>>>(bsum, nb);
  chunk_scan_kernel<<<(unsigned)nb, kThreads, 0, st>>>(cnt, nkeys, bsum);
  tile_starts_kernel<<<(g.ntiles + 256) / 256, 256, 0, st>>>(cnt, g.tlog, g.ntiles, sp.n,
                                                                     tile_off);
  c->launches += 5;
  return cudaGetLastError();
}

}  // namespace

hv_status sort_species(hv_ctx *c, int sidx, cudaStream_t stream) {
  Species &sp = c->sp[sidx];
  if (sp.n <= 1) return HV_OK;
  int32_t *cnt, *bsum, *rank;
  hv_status st = bucket_reserve(c, sp, &cnt, &bsum, &rank);
  if (st != HV_OK) return st;
  cudaError_t e = key_offsets(c, sp, cnt, bsum, rank, sp.tile_off, stream);
  if (e != cudaSuccess) return cuda_fail(e, "sort counts");
  // one ion per thread: every ion's loads are in flight at once
  const int blocks = (int)std::max<int64_t>((sp.n + 255) / 256, 1);
  bucket_scatter_kernel<<<blocks, 256, 0, stream>>>(c->g, sp.buf[sp.cur], sp.buf[sp.cur ^ 1],
                                                           sp.n, cnt, rank);
  c->launches++;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "sort");
  sp.cur ^= 1;
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
    sp.bucket = nullptr;
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
constexpr int kNoAllocMaxDevices = 64;

// About 16.3 MB of device memory per GPU.
static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocWords];

std::mutex g_noalloc_mu;
int32_t *g_noalloc_base[kNoAllocMaxDevices];

// Device address of the static scratch on the current device, looked up once
// per device (the first call on a device does this).
hv_status noalloc_base(int32_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "hv_sort_keys_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(HV_EINVAL, "hv_sort_keys_noalloc: device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_base[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return cuda_fail(e, "hv_sort_keys_noalloc: cudaGetSymbolAddress of the static scratch");
    g_noalloc_base[dev] = static_cast<int32_t *>(p);
  }
  *out = g_noalloc_base[dev];
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
