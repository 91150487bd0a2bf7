// In-repo device primitives: exclusive scan and a stable LSD radix sort
// (8-bit digits, per-tile histograms, warp-ballot ranking, shared-memory staging
// so that the scatter writes whole digit runs). Written for sm_103a; no CUB.
#pragma once

#include "common.cuh"

namespace dbbc {

// ------------------------------------------------------------------ scans
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Inclusive warp scan.
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(kFullMask, x, o);
    if ((int)lane_id() >= o) x += y;
  }
  return x;
}

// Exclusive block scan of one value per thread (blockDim.x == THREADS, a
// multiple of 32, at most 1024). Returns the exclusive prefix; *total gets the
// block sum. Contains __syncthreads.
template <typename T, int THREADS>
__device__ __forceinline__ T block_excl_scan(T x, T* total) {
  __shared__ T warp_tot[THREADS / 32];
  const int w = threadIdx.x >> 5;
  T inc = warp_incl_scan(x);
  if (lane_id() == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    T t = lane_id() < THREADS / 32 ? warp_tot[lane_id()] : T(0);
    T ti = warp_incl_scan(t);
    if (lane_id() < THREADS / 32) warp_tot[lane_id()] = ti - t;
    if (lane_id() == THREADS / 32 - 1) *total = ti;  // caller's shared slot
  }
  __syncthreads();
  return warp_tot[w] + inc - x;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const TI* in, int64_t n, TO* tile_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  TO s = 0;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    const int64_t k = base + i;
    if (k < n) s += (TO)in[k];
  }
  __shared__ TO tot;
  block_excl_scan<TO, kScanThreads>(s, &tot);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// In-place exclusive scan of the tile sums by one block of 1024 threads.
template <typename TO>
__global__ void __launch_bounds__(1024) scan_top_kernel(TO* sums, int64_t n, TO* grand_total) {
  __shared__ TO tot;
  TO carry = 0;
  for (int64_t base = 0; base < n; base += 1024) {
    const int64_t k = base + threadIdx.x;
    TO x = k < n ? sums[k] : TO(0);
    TO ex = block_excl_scan<TO, 1024>(x, &tot);
    if (k < n) sums[k] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && grand_total) *grand_total = carry;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) scan_down_kernel(const TI* in, int64_t n, const TO* tile_off,
                                                                 TO* out) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  TO v[kScanItems];
  TO s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    v[j] = (base + j < n) ? (TO)in[base + j] : TO(0);
    s += v[j];
  }
  __shared__ TO tot;
  TO run = block_excl_scan<TO, kScanThreads>(s, &tot) + tile_off[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
}

// out[i] = sum_{k<i} in[k]; optionally the grand total into device *total.
// `out` may alias `in`.
template <typename TI, typename TO>
void exclusive_scan(const TI* in, TO* out, int64_t n, cudaStream_t s, Scratch& scratch, TO* total = nullptr) {
  if (n <= 0) {
    if (total) DBBC_CUDA(cudaMemsetAsync(total, 0, sizeof(TO), s));
    return;
  }
  const int64_t tiles = ceil_div<int64_t>(n, kScanTile);
  TO* sums = scratch.get<TO>((size_t)tiles);
  scan_reduce_kernel<TI, TO><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums);
  DBBC_LAUNCH_CHECK();
  scan_top_kernel<TO><<<1, 1024, 0, s>>>(sums, tiles, total);
  DBBC_LAUNCH_CHECK();
  scan_down_kernel<TI, TO><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, sums, out);
  DBBC_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ radix sort
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
#ifndef DBBC_RS_ITEMS
#define DBBC_RS_ITEMS 8
#endif
#ifndef DBBC_RS_MATCH
#define DBBC_RS_MATCH 0
#endif
constexpr int kRsItems = DBBC_RS_ITEMS;         // keys per thread
constexpr int kRsTile = kRsThreads * kRsItems;  // keys per tile (2048 by default)

template <typename K>
__device__ __forceinline__ uint32_t rs_digit(K key, int shift) {
  return (uint32_t)(key >> shift) & 0xFFu;
}

// The lanes of the warp whose d (a digit, or 256 for "no key") equals this
// lane's: one ballot per bit of d, each lane keeping the lanes that agree with
// it on that bit. Nine ballots and a few logic operations per key run the
// digit passes faster than one warp match instruction per key (the Chung-Lu
// 1M x 200k x 20M build: 4.08 -> 3.70 ms). DBBC_RS_MATCH=1 builds the match
// form.
__device__ __forceinline__ unsigned rs_peers(uint32_t d) {
#if DBBC_RS_MATCH
  return __match_any_sync(kFullMask, d);
#else
  unsigned peers = kFullMask;
#pragma unroll
  for (int b = 0; b < 9; b++) {
    const bool bit = (d >> b) & 1u;
    const unsigned bal = __ballot_sync(kFullMask, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
#endif
}

// Per-tile digit counts, digit-major: hist[d * ntiles + tile]. Every thread
// loads its kRsItems keys before counting any, so that each warp has kRsItems
// loads in flight at once.
template <typename K>
__global__ void __launch_bounds__(kRsThreads) radix_hist_kernel(const K* __restrict__ keys, int64_t n, int shift,
                                                                 uint32_t* hist, int64_t ntiles) {
  __shared__ uint32_t h[kRsWarps][256];
  const int w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kRsTile + threadIdx.x;
  K key[kRsItems];
#pragma unroll
  for (int j = 0; j < kRsItems; j++) {
    const int64_t k = base + j * kRsThreads;
    key[j] = k < n ? keys[k] : K(0);
  }
  for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&h[0][0])[i] = 0;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kRsItems; j++) {
    const uint32_t d = base + j * kRsThreads < n ? rs_digit(key[j], shift) : 256u;
    const unsigned peers = rs_peers(d);
    if (d < 256u && (int)lane_id() == 31 - __clz(peers)) h[w][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  uint32_t c = 0;
#pragma unroll
  for (int ww = 0; ww < kRsWarps; ww++) c += h[ww][threadIdx.x];
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = c;
}

// One digit pass of the stable sort. A tile's keys (and values) are loaded
// first, all kRsItems per thread in flight together; each warp then ranks its
// 256 keys in input order (digit peers per key, per-warp digit counters), the
// block turns the per-warp counts into tile positions, the tile is staged in
// shared memory in digit order, and written out as whole digit runs at the
// offsets of the scanned digit-major histogram.
template <typename K, typename V, bool HAS_V>
__global__ void __launch_bounds__(kRsThreads) radix_scatter_kernel(const K* __restrict__ kin, const V* __restrict__ vin,
                                                                    K* __restrict__ kout, V* __restrict__ vout,
                                                                    int64_t n, int shift, const uint32_t* offs,
                                                                    int64_t ntiles) {
  extern __shared__ __align__(16) unsigned char rs_smem[];
  K* sk = reinterpret_cast<K*>(rs_smem);
  V* sv = reinterpret_cast<V*>(sk + kRsTile);
  uint32_t* wh = reinterpret_cast<uint32_t*>(HAS_V ? (void*)(sv + kRsTile) : (void*)(sk + kRsTile));
  uint32_t* bstart = wh + kRsWarps * 256;
  uint32_t* gofs = bstart + 256;
  __shared__ uint32_t tot_sh;

  const int w = threadIdx.x >> 5;
  const unsigned lane = lane_id();
  const int64_t tile_base = (int64_t)blockIdx.x * kRsTile;
  const int64_t wbase = tile_base + (int64_t)w * (kRsItems * 32);
  K key[kRsItems];
  V val[kRsItems];
#pragma unroll
  for (int j = 0; j < kRsItems; j++) {
    const int64_t i = wbase + j * 32 + lane;
    const bool valid = i < n;
    key[j] = valid ? kin[i] : K(0);
    if (HAS_V) val[j] = valid ? vin[i] : V(0);
  }
  for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) wh[i] = 0;
  gofs[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  __syncthreads();

  // digits (256 = past the end) and their warp peers, independent per item
  unsigned peers[kRsItems];
#pragma unroll
  for (int j = 0; j < kRsItems; j++) {
    const uint32_t d = wbase + j * 32 + lane < n ? rs_digit(key[j], shift) : 256u;
    peers[j] = rs_peers(d);
  }
  // rank within the warp, item by item in input order
  const unsigned lt_mask = (1u << lane) - 1u;
  uint32_t loc[kRsItems];
#pragma unroll
  for (int j = 0; j < kRsItems; j++) {
    const uint32_t d = wbase + j * 32 + lane < n ? rs_digit(key[j], shift) : 256u;
    uint32_t pre = 0;
    if (d < 256u) pre = wh[w * 256 + d];
    __syncwarp();
    loc[j] = pre + __popc(peers[j] & lt_mask);
    if (d < 256u && (int)lane == 31 - __clz(peers[j])) wh[w * 256 + d] = pre + __popc(peers[j]);
    __syncwarp();
  }
  __syncthreads();
  {  // per digit: exclusive prefix over warps, then over digits
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kRsWarps; ww++) {
      const uint32_t c = wh[ww * 256 + d];
      wh[ww * 256 + d] = run;
      run += c;
    }
    const uint32_t ex = block_excl_scan<uint32_t, kRsThreads>(run, &tot_sh);
    bstart[d] = ex;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kRsItems; j++) {
    const bool valid = wbase + j * 32 + lane < n;
    const uint32_t d = valid ? rs_digit(key[j], shift) : 256u;
    const uint32_t pos = valid ? bstart[d] + wh[w * 256 + d] + loc[j] : 0u;
    if (valid && DBBC_CHECK(pos < (uint32_t)kRsTile)) {
      sk[pos] = key[j];
      if (HAS_V) sv[pos] = val[j];
    }
  }
  __syncthreads();
  const int64_t rem = n - tile_base;
  const int cnt = rem < kRsTile ? (int)rem : kRsTile;
#pragma unroll
  for (int j = 0; j < kRsItems; j++) {
    const int i = threadIdx.x + j * kRsThreads;
    if (i < cnt) {
      const K k = sk[i];
      const uint32_t d = rs_digit(k, shift);
      const int64_t g = (int64_t)gofs[d] + (i - (int64_t)bstart[d]);
      if (DBBC_CHECK(g >= 0 && g < n)) {
        kout[g] = k;
        if (HAS_V) vout[g] = sv[i];
      }
    }
  }
}

template <typename K, typename V, bool HAS_V>
size_t radix_scatter_smem() {
  return (size_t)kRsTile * (sizeof(K) + (HAS_V ? sizeof(V) : 0)) + (size_t)(kRsWarps * 256 + 512) * 4;
}

// Stable sort of keys (and values) by bits [begin_bit, end_bit). Sorts between
// the two buffers of each pair; returns true when the result ended in the
// *_alt buffers. n < 2^32.
template <typename K, typename V, bool HAS_V>
bool radix_sort(K* keys, K* keys_alt, V* vals, V* vals_alt, int64_t n, int begin_bit, int end_bit, cudaStream_t s,
                Scratch& scratch) {
  if (n <= 1 || end_bit <= begin_bit) return false;
  const int64_t ntiles = ceil_div<int64_t>(n, kRsTile);
  uint32_t* hist = scratch.get<uint32_t>((size_t)ntiles * 256);
  const size_t smem = radix_scatter_smem<K, V, HAS_V>();
  DBBC_CUDA(cudaFuncSetAttribute(radix_scatter_kernel<K, V, HAS_V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  bool alt = false;
  for (int shift = begin_bit; shift < end_bit; shift += 8) {
    const K* kin = alt ? keys_alt : keys;
    K* kout = alt ? keys : keys_alt;
    const V* vin = alt ? vals_alt : vals;
    V* vout = alt ? vals : vals_alt;
    radix_hist_kernel<K><<<(unsigned)ntiles, kRsThreads, 0, s>>>(kin, n, shift, hist, ntiles);
    DBBC_LAUNCH_CHECK();
    exclusive_scan<uint32_t, uint32_t>(hist, hist, ntiles * 256, s, scratch);
    radix_scatter_kernel<K, V, HAS_V><<<(unsigned)ntiles, kRsThreads, smem, s>>>(kin, vin, kout, vout, n, shift,
                                                                                  hist, ntiles);
    DBBC_LAUNCH_CHECK();
    alt = !alt;
  }
  return alt;
}

}  // namespace dbbc
