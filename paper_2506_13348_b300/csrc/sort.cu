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
#include <mutex>

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
// sub-range [w * 32 R, (w+1) * 32 R), processed in R rounds of 32.  Two
// forms: the large 32-bit pair sort runs separate histogram, scan and
// scatter launches per pass with R = 16; sorts of up to 2^18 keys and every
// 64-bit (depth) sort run one kernel per pass (below) with R = 4 (small) or
// R = 8 (large 64-bit keys), so that enough blocks exist to fill the GPU.
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
  // the lanes sharing each element's digit, kept for the placement below
  unsigned pr[RS_ROUNDS];
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int idx = wbase + r * 32 + lane;
    const bool ok = idx < n;
    const uint32_t d = digit_of(kr[r], shift, mask);
    pr[r] = digit_peers(d, bits, ok);
    if (ok && (pr[r] & lt_mask) == 0) whist[warp][d] += __popc(pr[r]);
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
    const unsigned peers = pr[r];
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

// ---- one kernel per pass ("onesweep"): the small and the 64-bit sorts --------
// A first kernel counts the digits of every pass over all keys (one read of
// the keys); each pass then takes blocks of consecutive keys in the order the
// blocks start (an atomic ticket), ranks the block's keys by digit, publishes
// the block's digit counts and adds up those of all earlier blocks by a
// decoupled look-back over their published values, and writes the block's
// keys grouped by digit.  For the per-splat depth sort this replaces the
// histogram, scan and scatter launches of every pass by one launch; the
// large 32-bit pair sort keeps the separate passes, which measured faster
// there.
// A block waits only on blocks that took a smaller ticket, hence started
// earlier and are resident or done; every wait is bounded and a wait that
// runs out sets a device error flag (read by the host at its next
// synchronisation) and keeps its writes in bounds instead of hanging.
constexpr int RS_MAX_PASSES = 6;
constexpr uint32_t LB_AGG = 1u << 30, LB_PRE = 2u << 30, LB_VAL = (1u << 30) - 1u;
constexpr int LB_SPIN_LIMIT = 1 << 20;

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

struct SortPlan {
  int passes, step, begin, end;
  int bits(int p) const { return min(step, end - (begin + p * step)); }
  int shift(int p) const { return begin + p * step; }
};
static SortPlan sort_plan(int begin_bit, int end_bit) {
  // as few passes as 8-bit digits need, with the bits spread evenly over them
  // (e.g. 12 bits -> 2 x 6: fewer digits per pass means longer runs per block)
  SortPlan pl;
  pl.begin = begin_bit;
  pl.end = end_bit;
  pl.passes = (end_bit - begin_bit + 7) / 8;
  pl.step = pl.passes ? (end_bit - begin_bit + pl.passes - 1) / pl.passes : 1;
  return pl;
}

// digit counts of every pass: per block in shared memory, then one global
// atomic per non-zero bin
template <typename K, int R>
__global__ void __launch_bounds__(RS_THREADS) k_os_hist(const K* __restrict__ keys, int n, int begin, int step,
                                                         int end, int passes, uint32_t* __restrict__ ghist) {
  __shared__ uint32_t hist[RS_MAX_PASSES][RADIX];
  for (int i = threadIdx.x; i < RS_MAX_PASSES * RADIX; i += RS_THREADS) (&hist[0][0])[i] = 0;
  __syncthreads();
  constexpr int TILE = RS_THREADS * R;
  const int base = blockIdx.x * TILE;
  for (int i = threadIdx.x; i < TILE; i += RS_THREADS) {
    const int idx = base + i;
    if (idx >= n) break;
    const K k = keys[idx];
    for (int p = 0; p < passes; ++p) {
      const int sh = begin + p * step, bits = min(step, end - sh);
      atomicAdd(&hist[p][digit_of(k, sh, (1u << bits) - 1u)], 1u);
    }
  }
  __syncthreads();
  for (int p = 0; p < passes; ++p) {
    const int nd = 1 << min(step, end - (begin + p * step));
    for (int d = threadIdx.x; d < nd; d += RS_THREADS)
      if (hist[p][d]) atomicAdd(ghist + p * RADIX + d, hist[p][d]);
  }
}

template <typename K, int R>
__global__ void __launch_bounds__(RS_THREADS) k_os_pass(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                        K* __restrict__ kout, uint32_t* __restrict__ vout, int n,
                                                        int shift, int bits, const uint32_t* __restrict__ ghist,
                                                        uint32_t* __restrict__ status, uint32_t* __restrict__ ticket,
                                                        int* __restrict__ err) {
  constexpr int TILE = RS_THREADS * R, WARP_N = 32 * R;
  __shared__ uint32_t whist[RS_WARPS][RADIX];
  __shared__ K s_key[TILE];
  __shared__ uint32_t s_val[TILE];
  __shared__ uint32_t s_dstart[RADIX];
  __shared__ uint32_t s_goff[RADIX];
  __shared__ uint32_t s_wsum[RS_WARPS];
  __shared__ uint32_t s_gsum[RS_WARPS];
  __shared__ int s_bid;
  const uint32_t mask = (1u << bits) - 1u;
  const int nd = 1 << bits;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_bid = (int)atomicAdd(ticket, 1u);
  for (int i = lane; i < RADIX; i += 32) whist[warp][i] = 0;
  __syncthreads();
  const int bid = s_bid;
  const int wbase = bid * TILE + warp * WARP_N;
  K kr[R];
  uint32_t vr[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int idx = wbase + r * 32 + lane;
    kr[r] = idx < n ? kin[idx] : K(0);
    vr[r] = idx < n ? vin[idx] : 0u;
  }
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int idx = wbase + r * 32 + lane;
    const bool ok = idx < n;
    const uint32_t d = digit_of(kr[r], shift, mask);
    const unsigned peers = digit_peers(d, bits, ok);
    if (ok && (peers & lt_mask) == 0) whist[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit (thread dt): the warps' runs inside the block's run, the
  // block's count; the exclusive scans over digits of the block counts and
  // of the global counts
  const int dt = threadIdx.x;  // RS_THREADS == RADIX
  uint32_t cnt = 0, gcnt = 0;
  if (dt < nd) {
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
      const uint32_t c = whist[w][dt];
      whist[w][dt] = cnt;
      cnt += c;
    }
    gcnt = ghist[dt];
    // publish this block's count at once: later blocks can go on
    st_release(status + (size_t)bid * RADIX + dt, (bid == 0 ? LB_PRE : LB_AGG) | cnt);
  }
  uint32_t incl = cnt, gincl = gcnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o), u = __shfl_up_sync(0xffffffffu, gincl, o);
    if (lane >= o) {
      incl += t;
      gincl += u;
    }
  }
  if (lane == 31) {
    s_wsum[warp] = incl;
    s_gsum[warp] = gincl;
  }
  __syncthreads();
  uint32_t before = 0, gbefore = 0;
#pragma unroll
  for (int w = 0; w < RS_WARPS; ++w) {
    before += (w < warp) ? s_wsum[w] : 0u;
    gbefore += (w < warp) ? s_gsum[w] : 0u;
  }
  s_dstart[dt] = before + incl - cnt;
  // decoupled look-back, one thread per digit: the counts of digit dt in
  // all earlier blocks, back to the nearest block with a published prefix
  if (dt < nd) {
    uint32_t excl = 0;
    if (bid > 0) {
      int j = bid - 1, spins = 0;
      for (;;) {
        const uint32_t v = ld_acquire(status + (size_t)j * RADIX + dt);
        const uint32_t fl = v & ~LB_VAL;
        if (fl == 0u) {
          if (++spins > LB_SPIN_LIMIT) {
            atomicExch(err, 1);
            break;
          }
          __nanosleep(32);
          continue;
        }
        excl += v & LB_VAL;
        if (fl == LB_PRE || j == 0) break;
        --j;
      }
      st_release(status + (size_t)bid * RADIX + dt, LB_PRE | (excl + cnt));
    }
    s_goff[dt] = (gbefore + gincl - gcnt) + excl;  // global start of digit dt + earlier blocks
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < R; ++r) {
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
  const int nblk = min(TILE, n - bid * TILE);
  for (int sl = threadIdx.x; sl < nblk; sl += RS_THREADS) {
    const K key = s_key[sl];
    const uint32_t dd = digit_of(key, shift, mask);
    const uint32_t pos = s_goff[dd] + ((uint32_t)sl - s_dstart[dd]);
    if (pos < (uint32_t)n) {  // always, unless a look-back ran out (then the flag is set)
      kout[pos] = key;
      vout[pos] = s_val[sl];
    }
  }
}
static_assert(RS_THREADS == RADIX, "one thread per digit in the local scans");

// Temporaries: global digit counts, the look-back words (per pass, block and
// digit) and the tickets; one memset clears them all.
static size_t os_layout(int n, int nbits, size_t* status_off, size_t* ticket_off, int* nb_out) {
  const int tile = RS_THREADS * (n <= RS_SMALL_N ? 4 : 8);  // 64-bit keys past RS_SMALL_N: 2048 per block
  const int nb = ceil_div(n > 0 ? n : 1, tile);
  const int passes = std::max(1, (nbits + 7) / 8);
  const size_t ghist = (size_t)RS_MAX_PASSES * RADIX * 4;
  const size_t status = (size_t)passes * nb * RADIX * 4;
  *status_off = ghist;
  *ticket_off = ghist + status;
  if (nb_out) *nb_out = nb;
  return ghist + status + 256;
}

// The flags are a module variable (static device memory, one per device
// context, zero at load): taking them allocates nothing, which the
// no-allocation render relies on.  Word SORT_FLAG_LISTS: the depth order or
// a list derived from it may be wrong; word SORT_FLAG_ORDER: a rasteriser
// launch order may be wrong (the rasterisers then take the tiles in tile
// order, which changes no result).
__device__ int g_sort_err_flag[2];

namespace {
std::mutex g_err_mu;
int* g_sort_err[64] = {nullptr};
}  // namespace

int* sort_error_flag(int device) {
  if (device < 0 || device >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!g_sort_err[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_sort_err_flag) != cudaSuccess) return nullptr;  // the address of word 0
    g_sort_err[device] = static_cast<int*>(p);
  }
  return g_sort_err[device];
}

// Self-test of the bounded wait: one pass whose only block takes ticket 1,
// so the block it waits on (ticket 0) never runs and its look-back runs out.
// Returns 1 if the error flag came back set (and clears it), 0 if not, -1 on
// a CUDA error.
int sort_wait_selftest(cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  int* err = sort_error_flag(dev);
  if (!err) return -1;
  const int n = 2 * RS_THREADS * 4;  // two blocks' worth of keys
  size_t status_off, ticket_off;
  int nb;
  const size_t tb = os_layout(n, 6, &status_off, &ticket_off, &nb);
  char* buf = nullptr;
  const size_t kv = (size_t)n * 4;
  if (cudaMallocAsync(reinterpret_cast<void**>(&buf), tb + 4 * kv, st) != cudaSuccess) return -1;
  uint32_t* keys = reinterpret_cast<uint32_t*>(buf + tb);
  cudaMemsetAsync(buf, 0, tb + 4 * kv, st);
  const uint32_t one = 1;
  cudaMemcpyAsync(buf + ticket_off, &one, 4, cudaMemcpyHostToDevice, st);
  k_os_hist<uint32_t, 4><<<nb, RS_THREADS, 0, st>>>(keys, n, 0, 6, 6, 1, reinterpret_cast<uint32_t*>(buf));
  k_os_pass<uint32_t, 4><<<1, RS_THREADS, 0, st>>>(keys, keys + n, keys + 2 * n, keys + 3 * n, n, 0, 6,
                                                   reinterpret_cast<uint32_t*>(buf),
                                                   reinterpret_cast<uint32_t*>(buf + status_off),
                                                   reinterpret_cast<uint32_t*>(buf + ticket_off), err);
  note_launches(2);
  int h = 0;
  cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaMemsetAsync(err, 0, sizeof(int), st);
  cudaFreeAsync(buf, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
  return h ? 1 : 0;
}

template <typename K, int R>
static int radix_sort_os(K* k0, uint32_t* v0, K* k1, uint32_t* v1, int n, int begin_bit, int end_bit, void* temp,
                         cudaStream_t st, int flag_word) {
  if (n <= 1 || end_bit <= begin_bit) return 0;
  const SortPlan pl = sort_plan(begin_bit, end_bit);
  size_t status_off, ticket_off;
  int nb;
  const size_t bytes = os_layout(n, end_bit - begin_bit, &status_off, &ticket_off, &nb);
  char* t = reinterpret_cast<char*>(temp);
  uint32_t* ghist = reinterpret_cast<uint32_t*>(t);
  uint32_t* status = reinterpret_cast<uint32_t*>(t + status_off);
  uint32_t* tickets = reinterpret_cast<uint32_t*>(t + ticket_off);
  int dev = 0;
  cudaGetDevice(&dev);
  int* err = sort_error_flag(dev) + flag_word;
  cudaMemsetAsync(temp, 0, bytes, st);
  k_os_hist<K, R><<<nb, RS_THREADS, 0, st>>>(k0, n, pl.begin, pl.step, pl.end, pl.passes, ghist);
  note_launches(1);
  int cur = 0;
  K* kb[2] = {k0, k1};
  uint32_t* vb[2] = {v0, v1};
  for (int p = 0; p < pl.passes; ++p) {
    k_os_pass<K, R><<<nb, RS_THREADS, 0, st>>>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], n, pl.shift(p),
                                               pl.bits(p), ghist + p * RADIX, status + (size_t)p * nb * RADIX,
                                               tickets + p, err);
    note_launches(1);
    cur ^= 1;
  }
  return cur;
}

size_t radix_temp_bytes(int n, int key_bytes) {
  const int nb = ceil_div(n > 0 ? n : 1, rs_tile(n));
  const size_t cnt = (size_t)RADIX * nb;
  const size_t passes_path = 2 * cnt * sizeof(uint32_t) + 512 + scan_temp_bytes((int)cnt);
  if (key_bytes == 4 && n > RS_SMALL_N) return passes_path;  // the large 32-bit sort keeps separate passes
  size_t a, b;
  return std::max(passes_path, os_layout(n, 8 * RS_MAX_PASSES, &a, &b, nullptr));
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
    static_assert(sizeof(K) == 4, "the separate-pass sort is the 32-bit pair sort");
    k_radix_scatter_local<R><<<nb, RS_THREADS, 0, st>>>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], n, bit, bits,
                                                     offs, nb);
    note_launches(1);
    cur ^= 1;
  }
  return cur;
}

int radix_sort_u64(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1, int n, int begin_bit, int end_bit,
                   void* temp, cudaStream_t st) {
  // the per-splat depth sort: one kernel per pass at every size (at 12 M keys
  // 1.19 -> 0.98 ms against separate histogram / scan / scatter passes)
  if (n <= RS_SMALL_N)
    return radix_sort_os<uint64_t, 4>(k0, v0, k1, v1, n, begin_bit, end_bit, temp, st, SORT_FLAG_LISTS);
  return radix_sort_os<uint64_t, 8>(k0, v0, k1, v1, n, begin_bit, end_bit, temp, st, SORT_FLAG_LISTS);
}
int radix_sort_u32(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int n, int begin_bit, int end_bit,
                   void* temp, cudaStream_t st, int flag_word) {
  if (flag_word >= 0 && n <= RS_SMALL_N)
    return radix_sort_os<uint32_t, 4>(k0, v0, k1, v1, n, begin_bit, end_bit, temp, st, flag_word);
  return radix_sort_r<uint32_t, 16>(k0, v0, k1, v1, n, begin_bit, end_bit, temp, st);
}

// ---------------------------------------------------------------------------
// counts in depth order; an id out of range (only after a depth sort whose
// bounded wait ran out, which set the flag the host reads next) counts 0
__global__ void k_gather_counts(const uint32_t* __restrict__ order, const uint32_t* __restrict__ counts,
                                uint32_t* __restrict__ out, int n, int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t o = order[i];
  if (o < (uint32_t)n) {
    out[i] = counts[o];
  } else {
    out[i] = 0u;
    if (err) atomicExch(err + SORT_FLAG_LISTS, 1);
  }
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
    int dev = 0;
    cudaGetDevice(&dev);
    k_gather_counts<<<ceil_div(n, 256), 256, 0, st>>>(order, counts, counts_sorted, n, sort_error_flag(dev));
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
  constexpr unsigned FULL = 0xffffffffu;
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int first = warp_global * 32;
  if (first >= n) return;
  // lane l holds splat first + l (depth order); its pairs follow those of the
  // lanes before it, so the warp writes one contiguous run of pairs
  const int my = first + lane;
  uint32_t my_cnt = 0, my_item = 0, my_t0 = 0, my_w = 1, my_base = 0;
  if (my < n) {
    my_cnt = counts_sorted[my];
    if (my_cnt && order[my] >= (uint32_t)n) my_cnt = 0;  // see k_gather_counts: never, with the flag clear
    if (my_cnt) {
      my_item = order[my];
      const int4 rc = rects[my_item];
      const ViewDesc& V = vt.v[find_view_item(vt, (int)my_item)];
      my_t0 = (uint32_t)(V.tile_off + rc.z * V.tiles_x + rc.x);
      my_w = (uint32_t)(rc.y - rc.x + 1);
      my_base = (uint32_t)V.tiles_x;
    }
  }
  const uint32_t off0 = __shfl_sync(FULL, my < n ? offsets[my] : 0u, 0);
  // inclusive prefix of the counts over the warp
  uint32_t incl = my_cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += t;
  }
  const uint32_t total = __shfl_sync(FULL, incl, 31);
  // the warp writes its pairs 32 at a time: pair p's splat is the first lane
  // whose inclusive prefix exceeds p (binary search over the prefixes; for
  // p >= total the search stays in range and nothing is written)
  for (uint32_t base = 0; base < total; base += 32) {  // warp-uniform
    const uint32_t p = base + lane;
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const uint32_t v = __shfl_sync(FULL, incl, lo + step - 1);
      if (v <= p) lo += step;
    }
    const int s = lo;  // the number of lanes whose prefix is <= p
    const uint32_t start = __shfl_sync(FULL, incl - my_cnt, s);
    const uint32_t w = __shfl_sync(FULL, my_w, s), t0 = __shfl_sync(FULL, my_t0, s);
    const uint32_t tx = __shfl_sync(FULL, my_base, s), item = __shfl_sync(FULL, my_item, s);
    if (p < total) {
      const uint32_t k = p - start, row = k / w, col = k - row * w;
      tile_keys[off0 + p] = t0 + row * tx + col;
      pair_items[off0 + p] = item;
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
// A tile id out of range is skipped and raises the list flag (it cannot occur
// with the stable pair sort, which has no bounded wait).
__global__ void k_tile_ranges(const uint32_t* __restrict__ keys, int K, int n_tiles, uint2* __restrict__ ranges,
                              int* __restrict__ err) {
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
    if (t >= (uint32_t)n_tiles) {
      if (err) atomicExch(err + SORT_FLAG_LISTS, 1);
      continue;
    }
    if (i == 0 || k[j] != t) ranges[t].x = (uint32_t)i;
    if (i == K - 1 || k[2 + j] != t) ranges[t].y = (uint32_t)(i + 1);
  }
}

void launch_tile_ranges(const uint32_t* tile_keys, int K, int n_tiles, uint2* ranges, cudaStream_t st) {
  if (K > 0) {
    const int threads = (int)((K + 3) / 4);
    int dev = 0;
    cudaGetDevice(&dev);
    k_tile_ranges<<<ceil_div(threads, 256), 256, 0, st>>>(tile_keys, K, n_tiles, ranges, sort_error_flag(dev));
    note_launches(1);
  }
}

// Launch order of the rasterisers' tiles: longest list first.  The key is an
// 8-bit code of the list length (exact below 8, then exponent and three
// mantissa bits, so within 12.5 %), inverted for a descending sort; the
// stable sort keeps tile order among equal codes.  Issued in this order the
// tiles with the most entries start in the grid's first wave instead of
// stretching its last one.
__device__ __forceinline__ uint32_t length_code(uint32_t len) {
  if (len < 8u) return len;
  const int e = 31 - __clz((int)len);                         // 3..31
  return ((uint32_t)(e - 2) << 3) | ((len >> (e - 3)) & 7u);  // 8..239
}

__global__ void k_tile_order_keys(const uint2* __restrict__ ranges, int n, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ ids) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint2 r = ranges[i];
  keys[i] = 255u - length_code(r.y - r.x);
  ids[i] = (uint32_t)i;
}

// Backward variant: the entries the backward walks in a tile, i.e. up to the
// last blended entry of its pixels (saved by the forward), instead of the
// whole list.  One CTA of 256 threads per tile, one thread per pixel.
__global__ void __launch_bounds__(256) k_tile_walk_keys(ViewTable vt, const uint2* __restrict__ ranges,
                                                        uint32_t* __restrict__ keys, uint32_t* __restrict__ ids) {
  const int tile = blockIdx.x;
  const ViewDesc& V = vt.v[find_view(vt, tile)];
  const int tl = tile - V.tile_off;
  const int px = (tl % V.tiles_x) * TILE + (threadIdx.x & (TILE - 1));
  const int py = (tl / V.tiles_x) * TILE + (threadIdx.x / TILE);
  const uint2 r = ranges[tile];
  uint32_t walk = 0;
  if (px < V.W && py < V.H) {
    const int last = V.last[py * V.W + px];
    if (last >= (int)r.x) walk = (uint32_t)last - r.x + 1u;
  }
  walk = __reduce_max_sync(0xffffffffu, walk);
  __shared__ uint32_t s_w[8];
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = walk;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) m = max(m, s_w[w]);
    keys[tile] = 255u - length_code(m);
    ids[tile] = (uint32_t)tile;
  }
}

const uint32_t* launch_tile_order_walk(const ViewTable& vt, const uint2* ranges, uint32_t* buf, void* temp,
                                       cudaStream_t st) {
  const int n = vt.n_tiles;
  if (n <= 0) return buf + n;
  k_tile_walk_keys<<<n, 256, 0, st>>>(vt, ranges, buf, buf + n);
  note_launches(1);
  const int w = radix_sort_u32(buf, buf + n, buf + 2 * n, buf + 3 * n, n, 0, 8, temp, st, SORT_FLAG_ORDER);
  return w ? buf + 3 * n : buf + n;
}

const uint32_t* launch_tile_order(const uint2* ranges, int n, uint32_t* buf, void* temp, cudaStream_t st) {
  if (n <= 0) return buf + n;
  k_tile_order_keys<<<ceil_div(n, 256), 256, 0, st>>>(ranges, n, buf, buf + n);
  note_launches(1);
  const int w = radix_sort_u32(buf, buf + n, buf + 2 * n, buf + 3 * n, n, 0, 8, temp, st, SORT_FLAG_ORDER);
  return w ? buf + 3 * n : buf + n;
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
