// Binning and sorting: exclusive scan, stable LSD radix sort, pair emission
// and per-tile ranges.
//
// Order of work (per batch of views):
//   1. splats are sorted once by (view, depth bits) -- N items, 32 + view bits;
//   2. the (tile, item) pairs are emitted in that order;
//   3. the pairs are stably sorted by global tile id only (ceil(log2 tiles)
//      bits, 2 passes for up to 65536 tiles).
// Stability of step 3 keeps the depth order (and the item-id order for equal
// depths) inside each tile, so the result equals a sort of 64-bit
// (tile << 32 | depth bits) keys with ties by item id, at a fraction of the
// traffic: 8-byte pairs over 2 passes instead of 12-byte pairs over 6.
#include <algorithm>

#include "kernels.h"
#include "prof.h"

namespace ts {

constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 4;  // per thread
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

// Block-wide exclusive scan of SCAN_TILE u32 values; writes block sum.
__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_tiles(const uint32_t* __restrict__ in,
                                                            uint32_t* __restrict__ out, int n,
                                                            uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t warp_sums[SCAN_BLOCK / 32];
  const int base = blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  uint32_t local = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0u;
    local += v[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t ws = warp_sums[lane];
    uint32_t wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    warp_sums[lane] = wi - ws;
    if (lane == 31 && block_sums) block_sums[blockIdx.x] = wi;
  }
  __syncthreads();
  uint32_t run = warp_sums[warp] + incl - local;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int n, const uint32_t* __restrict__ block_offs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += block_offs[i / SCAN_TILE];
}

static int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

size_t scan_temp_bytes(int n) {
  size_t total = 0;
  while (n > SCAN_TILE) {
    n = ceil_div(n, SCAN_TILE);
    total += 2 * (size_t)n * sizeof(uint32_t) + 256;
  }
  return total + 256;
}

void launch_exclusive_scan(const uint32_t* in, uint32_t* out, int n, void* temp, cudaStream_t st) {
  if (n <= 0) return;
  const int nb = ceil_div(n, SCAN_TILE);
  if (nb == 1) {
    k_scan_tiles<<<1, SCAN_BLOCK, 0, st>>>(in, out, n, nullptr);
    note_launches(1);
    return;
  }
  uint32_t* sums = reinterpret_cast<uint32_t*>(temp);
  uint32_t* offs = sums + nb;
  char* rest = reinterpret_cast<char*>(offs + nb);
  rest = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(rest) + 255) & ~uintptr_t(255));
  k_scan_tiles<<<nb, SCAN_BLOCK, 0, st>>>(in, out, n, sums);
  note_launches(1);
  launch_exclusive_scan(sums, offs, nb, rest, st);
  k_scan_add<<<ceil_div(n, 256), 256, 0, st>>>(out, n, offs);
  note_launches(1);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort, digits of at most 8 bits.
// A block owns 256 * R consecutive keys; warp w of the block owns the
// sub-range [w * 32 R, (w+1) * 32 R), processed in R rounds of 32.  Small
// sorts (the per-splat depth sort) take R = 4 so that enough blocks exist
// to fill the GPU; the pair sort takes R = 16.
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RADIX = 256;
constexpr int RS_SMALL_N = 1 << 18;
template <int R>
struct RsTile {
  static constexpr int WARP = 32 * R;
  static constexpr int N = RS_WARPS * WARP;
};
static int rs_tile(int n) { return n <= RS_SMALL_N ? RsTile<4>::N : RsTile<16>::N; }

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K key, int shift, uint32_t mask) {
  return (uint32_t)(key >> shift) & mask;
}

// Lanes of the warp holding the same digit (and a valid element): one ballot
// per digit bit, cheaper than a general match for digits of <= 8 bits.
__device__ __forceinline__ unsigned digit_peers(uint32_t d, int bits, bool ok) {
  unsigned peers = __ballot_sync(0xffffffffu, ok);
  for (int b = 0; b < bits; ++b) {
    const bool set = (d >> b) & 1u;
    const unsigned bb = __ballot_sync(0xffffffffu, set);
    peers &= set ? bb : ~bb;
  }
  return peers;
}

template <typename K, int R>
__global__ void __launch_bounds__(RS_THREADS) k_radix_hist(const K* __restrict__ keys, int n, int shift,
                                                            uint32_t mask, uint32_t* __restrict__ counts,
                                                            int nblocks) {
  __shared__ uint32_t hist[RADIX];
  for (int i = threadIdx.x; i < RADIX; i += RS_THREADS) hist[i] = 0;
  __syncthreads();
  constexpr int RS_TILE = RsTile<R>::N;
  const int base = blockIdx.x * RS_TILE;
  for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
    // plain shared-memory atomics (aggregating equal digits per warp first
    // with ballots or a match measured slower)
    const int idx = base + i;
    if (idx < n) atomicAdd(&hist[digit_of(keys[idx], shift, mask)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d <= (int)mask; d += RS_THREADS) counts[(size_t)d * nblocks + blockIdx.x] = hist[d];
}

template <typename K, int R>
__global__ void __launch_bounds__(RS_THREADS) k_radix_scatter(const K* __restrict__ kin,
                                                               const uint32_t* __restrict__ vin,
                                                               K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                               int n, int shift, uint32_t mask,
                                                               const uint32_t* __restrict__ offsets, int nblocks) {
  __shared__ uint32_t whist[RS_WARPS][RADIX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = lane; i < RADIX; i += 32) whist[warp][i] = 0;
  __syncwarp();
  constexpr int RS_ROUNDS = R;
  const int wbase = blockIdx.x * RsTile<R>::N + warp * RsTile<R>::WARP;
  K kr[RS_ROUNDS];
  uint32_t dg[RS_ROUNDS];
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int idx = wbase + r * 32 + lane;
    const bool ok = idx < n;
    kr[r] = ok ? kin[idx] : K(0);
    dg[r] = ok ? digit_of(kr[r], shift, mask) : 0xffffffffu;
    const unsigned peers = __match_any_sync(0xffffffffu, dg[r]);
    if (ok && (peers & lt_mask) == 0) whist[warp][dg[r]] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // exclusive prefix over warps, offset by the block's global digit offset
  for (int d = threadIdx.x; d <= (int)mask; d += RS_THREADS) {
    uint32_t run = offsets[(size_t)d * nblocks + blockIdx.x];
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      const uint32_t c = whist[w][d];
      whist[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int idx = wbase + r * 32 + lane;
    const bool ok = idx < n;
    const unsigned peers = __match_any_sync(0xffffffffu, dg[r]);
    uint32_t pos = 0;
    if (ok) {
      pos = whist[warp][dg[r]] + __popc(peers & lt_mask);
      kout[pos] = kr[r];
      vout[pos] = vin[idx];
    }
    __syncwarp();
    if (ok && (peers & lt_mask) == 0) whist[warp][dg[r]] += __popc(peers);
    __syncwarp();
  }
}

// Scatter with a block-local reorder (32-bit keys): the block first places
// its RS_TILE elements in shared memory grouped by digit (stable), then
// threads write consecutive slots, so each digit's run of the block goes out
// as consecutive addresses instead of one scattered 4-byte store per element.
template <int R>
__global__ void __launch_bounds__(RS_THREADS, 3) k_radix_scatter_local(const uint32_t* __restrict__ kin,
                                                                     const uint32_t* __restrict__ vin,
                                                                     uint32_t* __restrict__ kout,
                                                                     uint32_t* __restrict__ vout, int n, int shift,
                                                                     int bits,
                                                                     const uint32_t* __restrict__ offsets,
                                                                     int nblocks) {
  constexpr int RS_ROUNDS = R, RS_TILE = RsTile<R>::N;
  __shared__ uint32_t whist[RS_WARPS][RADIX];
  __shared__ uint32_t s_key[RS_TILE];
  __shared__ uint32_t s_val[RS_TILE];
  __shared__ uint32_t s_dstart[RADIX];
  __shared__ uint32_t s_goff[RADIX];
  __shared__ uint32_t s_wsum[RS_WARPS];
  const uint32_t mask = (1u << bits) - 1u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = lane; i < RADIX; i += 32) whist[warp][i] = 0;
  __syncwarp();
  const int wbase = blockIdx.x * RS_TILE + warp * RsTile<R>::WARP;
  // all loads of the warp's keys and values first (32 in flight per thread)
  uint32_t kr[RS_ROUNDS], vr[RS_ROUNDS];
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int idx = wbase + r * 32 + lane;
    kr[r] = idx < n ? kin[idx] : 0u;
    vr[r] = idx < n ? vin[idx] : 0u;
  }
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int idx = wbase + r * 32 + lane;
    const bool ok = idx < n;
    const uint32_t d = digit_of(kr[r], shift, mask);
    const unsigned peers = digit_peers(d, bits, ok);
    if (ok && (peers & lt_mask) == 0) whist[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: warp runs inside the block's run (exclusive over warps), the
  // block's count, then an exclusive scan of the counts over digits
  const int dt = threadIdx.x;  // RS_THREADS == RADIX
  uint32_t cnt = 0;
  if (dt <= (int)mask) {
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      const uint32_t c = whist[w][dt];
      whist[w][dt] = cnt;
      cnt += c;
    }
    s_goff[dt] = offsets[(size_t)dt * nblocks + blockIdx.x];
  }
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  uint32_t before = 0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) before += (w < warp) ? s_wsum[w] : 0u;
  s_dstart[dt] = before + incl - cnt;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int idx = wbase + r * 32 + lane;
    const bool ok = idx < n;
    const uint32_t d = digit_of(kr[r], shift, mask);
    const unsigned peers = digit_peers(d, bits, ok);
    if (ok) {
      const uint32_t slot = s_dstart[d] + whist[warp][d] + __popc(peers & lt_mask);
      s_key[slot] = kr[r];
      s_val[slot] = vr[r];
    }
    __syncwarp();
    if (ok && (peers & lt_mask) == 0) whist[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  const int nblk = min(RS_TILE, n - (int)blockIdx.x * RS_TILE);
  for (int sl = threadIdx.x; sl < nblk; sl += RS_THREADS) {
    const uint32_t key = s_key[sl];
    const uint32_t dd = digit_of(key, shift, mask);
    const uint32_t pos = s_goff[dd] + ((uint32_t)sl - s_dstart[dd]);
    kout[pos] = key;
    vout[pos] = s_val[sl];
  }
}
static_assert(RS_THREADS == RADIX, "one thread per digit in the local scan");

size_t radix_temp_bytes(int n) {
  const int nb = ceil_div(n > 0 ? n : 1, rs_tile(n));
  const size_t cnt = (size_t)RADIX * nb;
  return 2 * cnt * sizeof(uint32_t) + 512 + scan_temp_bytes((int)cnt);
}

template <typename K, int R>
static int radix_sort_r(K* k0, uint32_t* v0, K* k1, uint32_t* v1, int n, int begin_bit, int end_bit, void* temp,
                      cudaStream_t st) {
  if (n <= 1 || end_bit <= begin_bit) return 0;
  const int nb = ceil_div(n, RsTile<R>::N);
  const size_t cnt = (size_t)RADIX * nb;
  uint32_t* counts = reinterpret_cast<uint32_t*>(temp);
  uint32_t* offs = counts + cnt;
  char* rest = reinterpret_cast<char*>(offs + cnt);
  rest = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(rest) + 255) & ~uintptr_t(255));
  int cur = 0;
  K* kb[2] = {k0, k1};
  uint32_t* vb[2] = {v0, v1};
  // as few passes as 8-bit digits need, with the bits spread evenly over them
  // (e.g. 12 bits -> 2 x 6: fewer digits per pass means longer runs per block)
  const int passes = (end_bit - begin_bit + 7) / 8;
  const int step = (end_bit - begin_bit + passes - 1) / passes;
  for (int bit = begin_bit; bit < end_bit; bit += step) {
    const int bits = min(step, end_bit - bit);
    const uint32_t mask = (1u << bits) - 1u;
    const int nd = 1 << bits;
    k_radix_hist<K, R><<<nb, RS_THREADS, 0, st>>>(kb[cur], n, bit, mask, counts, nb);
    note_launches(1);
    launch_exclusive_scan(counts, offs, nd * nb, rest, st);
    if constexpr (sizeof(K) == 4)
      k_radix_scatter_local<R><<<nb, RS_THREADS, 0, st>>>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], n, bit, bits,
                                                       offs, nb);
    else
      k_radix_scatter<K, R><<<nb, RS_THREADS, 0, st>>>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], n, bit, mask, offs,
                                                    nb);
    note_launches(1);
    cur ^= 1;
  }
  return cur;
}

template <typename K>
static int radix_sort(K* k0, uint32_t* v0, K* k1, uint32_t* v1, int n, int begin_bit, int end_bit, void* temp,
                      cudaStream_t st) {
  if (n <= RS_SMALL_N) return radix_sort_r<K, 4>(k0, v0, k1, v1, n, begin_bit, end_bit, temp, st);
  return radix_sort_r<K, 16>(k0, v0, k1, v1, n, begin_bit, end_bit, temp, st);
}

int radix_sort_u64(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int n, int begin_bit, int end_bit,
                   void* temp, cudaStream_t st) {
  return radix_sort<uint64_t>(k0, v0, k1, v1, n, begin_bit, end_bit, temp, st);
}
int radix_sort_u32(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int n, int begin_bit, int end_bit,
                   void* temp, cudaStream_t st) {
  return radix_sort<uint32_t>(k0, v0, k1, v1, n, begin_bit, end_bit, temp, st);
}

// ---------------------------------------------------------------------------
__global__ void k_gather_counts(const uint32_t* __restrict__ order, const uint32_t* __restrict__ counts,
                                uint32_t* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = counts[order[i]];
}

// 64-bit total of the per-splat pair counts (the 32-bit scan would wrap past
// 2^32 pairs): one reduction per block, one atomic per block.
__global__ void __launch_bounds__(256) k_sum_counts(const uint32_t* __restrict__ counts, int n,
                                                    unsigned long long* __restrict__ total) {
  __shared__ unsigned long long part[8];
  unsigned long long s = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += counts[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < 8; ++w) t += part[w];
    if (t) atomicAdd(total, t);
  }
}

void launch_sum_counts(const uint32_t* counts, int n, unsigned long long* total, cudaStream_t st) {
  cudaMemsetAsync(total, 0, sizeof(unsigned long long), st);
  if (n > 0) {
    const int blocks = std::min(ceil_div(n, 256), 148 * 4);
    k_sum_counts<<<blocks, 256, 0, st>>>(counts, n, total);
    note_launches(1);
  }
}

void launch_gather_counts(const uint32_t* order, const uint32_t* counts, uint32_t* counts_sorted, int n,
                          cudaStream_t st) {
  if (n > 0) {
    k_gather_counts<<<ceil_div(n, 256), 256, 0, st>>>(order, counts, counts_sorted, n);
    note_launches(1);
  }
}

// One warp per 32 depth-sorted items; the warp writes each item's tile
// pairs in turn with coalesced stores (items differ a lot in tile count).
__global__ void __launch_bounds__(256) k_emit_pairs(ViewTable vt, const uint32_t* __restrict__ order,
                                                     const uint32_t* __restrict__ offsets,
                                                     const uint32_t* __restrict__ counts_sorted,
                                                     const int4* __restrict__ rects, uint32_t* __restrict__ tile_keys,
                                                     uint32_t* __restrict__ pair_items, int n) {
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int first = warp_global * 32;
  if (first >= n) return;
  const int my = first + lane;
  uint32_t my_item = 0, my_cnt = 0, my_off = 0;
  int4 my_rc = make_int4(0, 0, 0, 0);
  if (my < n) {
    my_cnt = counts_sorted[my];
    if (my_cnt) {
      my_item = order[my];
      my_off = offsets[my];
      my_rc = rects[my_item];  // loaded up front: the loop below has no dependent global loads
    }
  }
  unsigned todo = __ballot_sync(0xffffffffu, my_cnt != 0);
  while (todo) {
    const int src = __ffs(todo) - 1;
    todo &= todo - 1;
    const uint32_t item = __shfl_sync(0xffffffffu, my_item, src);
    const uint32_t cnt = __shfl_sync(0xffffffffu, my_cnt, src);
    const uint32_t off = __shfl_sync(0xffffffffu, my_off, src);
    const int v = find_view_item(vt, (int)item);
    const ViewDesc& V = vt.v[v];
    int4 rc;
    rc.x = __shfl_sync(0xffffffffu, my_rc.x, src);
    rc.y = __shfl_sync(0xffffffffu, my_rc.y, src);
    rc.z = __shfl_sync(0xffffffffu, my_rc.z, src);
    const int w = rc.y - rc.x + 1;
    // lane's tile (row, column) in the rect, advanced by 32 entries per step
    // without a division per entry
    int col = lane % w, row = lane / w;
    const int dq = 32 / w, dr = 32 % w;
    const uint32_t t0 = (uint32_t)(V.tile_off + rc.z * V.tiles_x + rc.x);
    for (uint32_t j = lane; j < cnt; j += 32) {
      tile_keys[off + j] = t0 + (uint32_t)(row * V.tiles_x + col);
      pair_items[off + j] = item;
      col += dr;
      row += dq;
      if (col >= w) {
        col -= w;
        ++row;
      }
    }
  }
}

void launch_emit_pairs(const ViewTable& vt, const uint32_t* order, const uint32_t* offsets,
                       const uint32_t* counts_sorted, const int4* rects, uint32_t* tile_keys,
                       uint32_t* pair_items, int n, cudaStream_t st) {
  if (n > 0) {
    k_emit_pairs<<<ceil_div(n, 256), 256, 0, st>>>(vt, order, offsets, counts_sorted, rects, tile_keys,
                                                  pair_items, n);
    note_launches(1);
  }
}

// Tile ranges from the sorted tile ids: 4 keys per thread (one 16-byte
// load plus the neighbours at both ends), a range boundary wherever the id
// changes.
__global__ void k_tile_ranges(const uint32_t* __restrict__ keys, int K, uint2* __restrict__ ranges) {
  const long long i0 = 4ll * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 >= K) return;
  uint32_t k[6];
  k[0] = i0 > 0 ? keys[i0 - 1] : 0xffffffffu;
  if (i0 + 4 <= K) {
    const uint4 q = *reinterpret_cast<const uint4*>(keys + i0);
    k[1] = q.x; k[2] = q.y; k[3] = q.z; k[4] = q.w;
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) k[1 + j] = (i0 + j < K) ? keys[i0 + j] : 0xffffffffu;
  }
  k[5] = (i0 + 4 < K) ? keys[i0 + 4] : 0xffffffffu;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const long long i = i0 + j;
    if (i >= K) break;
    const uint32_t t = k[1 + j];
    if (i == 0 || k[j] != t) ranges[t].x = (uint32_t)i;
    if (i == K - 1 || k[2 + j] != t) ranges[t].y = (uint32_t)(i + 1);
  }
}

void launch_tile_ranges(const uint32_t* tile_keys, int K, uint2* ranges, cudaStream_t st) {
  if (K > 0) {
    const int threads = (int)((K + 3) / 4);
    k_tile_ranges<<<ceil_div(threads, 256), 256, 0, st>>>(tile_keys, K, ranges);
    note_launches(1);
  }
}

__global__ void k_depth_bits(const uint64_t* __restrict__ dk, uint32_t* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const uint64_t k = dk[i];
    out[i] = (k == ~0ull) ? 0xffffffffu : (uint32_t)(k & 0xffffffffull);
  }
}

void launch_depth_bits(const uint64_t* depth_keys_unsorted, uint32_t* out, int n, cudaStream_t st) {
  if (n > 0) {
    k_depth_bits<<<ceil_div(n, 256), 256, 0, st>>>(depth_keys_unsorted, out, n);
    note_launches(1);
  }
}

}  // namespace ts
