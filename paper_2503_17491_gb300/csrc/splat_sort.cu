// K2-K4: tile binning.
//
// The per-tile lists sorted by range (Sec. 3.2.1) are built in three steps:
//   1. a stable radix sort of all (view, primitive) pairs by their binary32 range key
//      (one key per pair, not per tile: far fewer keys than (tile, primitive) entries);
//   2. emission, in that order, of one (global tile id, pair id) entry per touched tile, at
//      offsets given by an exclusive scan of the tile counts (K2);
//   3. a stable radix sort of the entries by tile id (K3).  Stability keeps step 1's order
//      inside every tile, so each list ends up in (tile, range, id) order -- the same order as
//      sorting 64-bit (tile << 32 | range bits) keys with the id as the final tie-break.
// Tile ranges [start, end) follow from the sorted tile ids (K4).
//
// The sort is a reduce-then-scan LSD radix sort with 8-bit digits on a fixed grid of CTAs, so
// that the element count can live on the device (it is data dependent after emission) and the
// whole pipeline can be captured in a CUDA graph.  Ranking inside a CTA tile is warp-level
// (match.any) and stable in (warp, item, lane) = index order; the ranked tile is first sorted
// by digit in shared memory and then written out run by run, so that global stores coalesce.

#include "splat_internal.cuh"

namespace splat {
namespace {

constexpr int kRadix = 256;
constexpr int kThreads = 256;
constexpr int kItems = kSortTile / kThreads;   // 8
constexpr int kWarps = kThreads / 32;

__device__ __forceinline__ int64_t chunk_of(int64_t n, int grid)
{
    int64_t c = (n + grid - 1) / grid;
    return (c + kSortTile - 1) / kSortTile * kSortTile;
}

__device__ __forceinline__ int64_t clamp_count(const uint32_t *d_count, int64_t max_n)
{
    int64_t n = d_count ? static_cast<int64_t>(*d_count) : max_n;
    return n < max_n ? n : max_n;
}

// per-CTA digit histogram: hist[digit * grid + cta]
__global__ void __launch_bounds__(kThreads) k_upsweep(const uint32_t *__restrict__ keys,
                                                      const uint32_t *d_count, int64_t max_n,
                                                      int shift, int drop_max,
                                                      uint32_t *__restrict__ hist)
{
    __shared__ uint32_t s_cnt[kWarps][kRadix];
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int k = tid; k < kWarps * kRadix; k += kThreads) (&s_cnt[0][0])[k] = 0;
    __syncthreads();
    const int64_t n = clamp_count(d_count, max_n);
    const int64_t chunk = chunk_of(n, gridDim.x);
    const int64_t begin = chunk * blockIdx.x;
    const int64_t end = begin + chunk < n ? begin + chunk : n;
    for (int64_t j = begin + tid; j < end; j += kThreads) {
        const uint32_t k = keys[j];
        if (!(drop_max && k == 0xFFFFFFFFu)) atomicAdd(&s_cnt[warp][(k >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += s_cnt[w][tid];
    hist[static_cast<int64_t>(tid) * gridDim.x + blockIdx.x] = t;
}

// per digit (one warp each): exclusive scan of its kSortGrid per-CTA counts hist[d * grid + b]
// in place, and the digit's total into dtot[d].  Each lane takes a run of kPer consecutive
// counts, so all loads are issued before the one warp scan of the run sums.
__global__ void __launch_bounds__(256) k_scan_digits(uint32_t *__restrict__ hist, int grid,
                                                     uint32_t *__restrict__ dtot)
{
    constexpr int kPer = (kSortGrid + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int d = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (d >= kRadix) return;
    uint32_t *h = hist + static_cast<int64_t>(d) * grid;
    uint32_t v[kPer];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int b = lane * kPer + i;
        v[i] = b < grid ? h[b] : 0u;
        sum += v[i];
    }
    uint32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    uint32_t run = x - sum;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int b = lane * kPer + i;
        if (b < grid) h[b] = run;
        run += v[i];
    }
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, x, 31);
    if (lane == 0) dtot[d] = total;
}

__global__ void __launch_bounds__(kThreads) k_downsweep(
    const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
    uint32_t *__restrict__ keys_out, uint32_t *__restrict__ vals_out, const uint32_t *d_count,
    int64_t max_n, int shift, int drop_max, const uint32_t *__restrict__ hist,
    const uint32_t *__restrict__ dtot, const uint64_t *__restrict__ aux_in,
    uint64_t *__restrict__ aux_out)
{
    __shared__ uint32_t s_base[kRadix];          // running global offset per digit
    __shared__ uint32_t s_wcnt[kWarps][kRadix];  // per-warp digit counts -> warp prefixes
    __shared__ uint32_t s_tile[kRadix];          // digit totals of the current tile
    __shared__ uint32_t s_toff[kRadix];          // digit offsets inside the current tile
    __shared__ uint32_t s_wsum[kWarps];
    __shared__ uint32_t s_kept;                  // items of the current tile that are written
    __shared__ uint32_t s_key[kSortTile], s_val[kSortTile];   // the tile, sorted by digit
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n = clamp_count(d_count, max_n);
    const int64_t chunk = chunk_of(n, gridDim.x);
    const int64_t begin = chunk * blockIdx.x;
    const int64_t end = begin + chunk < n ? begin + chunk : n;
    if (begin >= end) return;
    {   // digit base: exclusive scan of the digit totals, plus this CTA's offset in its digit
        const uint32_t t = dtot[tid];
        uint32_t x = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_tile[warp] = x;
        __syncthreads();
        uint32_t wbase = 0;
        for (int w = 0; w < warp; ++w) wbase += s_tile[w];
        s_base[tid] = wbase + x - t + hist[static_cast<int64_t>(tid) * gridDim.x + blockIdx.x];
        __syncthreads();
    }
    const uint32_t lt_mask = (1u << lane) - 1u;

    for (int64_t tb = begin; tb < end; tb += kSortTile) {
        for (int k = tid; k < kWarps * kRadix; k += kThreads) (&s_wcnt[0][0])[k] = 0;
        __syncthreads();
        uint32_t key[kItems], val[kItems], rank[kItems];
        int dig[kItems];
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            const int64_t j = tb + warp * (32 * kItems) + it * 32 + lane;
            key[it] = j < end ? keys_in[j] : 0u;
            const bool valid = j < end && !(drop_max && key[it] == 0xFFFFFFFFu);
            val[it] = valid ? vals_in[j] : 0u;
            dig[it] = valid ? static_cast<int>((key[it] >> shift) & 0xFF) : kRadix + lane;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, dig[it]);
            uint32_t before = 0;
            if (valid) before = s_wcnt[warp][dig[it]];
            __syncwarp();
            rank[it] = before + __popc(peers & lt_mask);
            const int last = 31 - __clz(peers);
            if (valid && lane == last) s_wcnt[warp][dig[it]] = before + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {   // digit tid: exclusive prefix over warps, tile total
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = s_wcnt[w][tid];
                s_wcnt[w][tid] = run;
                run += c;
            }
            s_tile[tid] = run;
            // the digit's offset inside the tile: exclusive scan of the tile totals over digits
            uint32_t x = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_wsum[warp] = x;
            __syncthreads();
            uint32_t wbase = 0;
            for (int w = 0; w < warp; ++w) wbase += s_wsum[w];
            s_toff[tid] = wbase + x - run;
            if (tid == kRadix - 1) s_kept = wbase + x;
        }
        __syncthreads();
        // sort the tile by digit in shared memory (stable: warp, item, lane order) ...
#pragma unroll
        for (int it = 0; it < kItems; ++it) {
            if (dig[it] < kRadix) {
                const uint32_t lpos = s_toff[dig[it]] + s_wcnt[warp][dig[it]] + rank[it];
                s_key[lpos] = key[it];
                s_val[lpos] = val[it];
            }
        }
        __syncthreads();
        // ... and write each digit's run to its global place: consecutive threads, consecutive
        // addresses
        const int cnt = static_cast<int>(s_kept);
        for (int i = tid; i < cnt; i += kThreads) {
            const uint32_t k = s_key[i];
            const int d = static_cast<int>((k >> shift) & 0xFF);
            const uint32_t pos = s_base[d] + (static_cast<uint32_t>(i) - s_toff[d]);
            keys_out[pos] = k;
            vals_out[pos] = s_val[i];
            if (aux_out) aux_out[pos] = aux_in[s_val[i]];
        }
        __syncthreads();
        s_base[tid] += s_tile[tid];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// emission (K2)
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ uint32_t rect_count(uint64_t w)
{
    return static_cast<uint32_t>((w >> 16) & 0xFFFFu) * static_cast<uint32_t>(w >> 48);
}

// per-CTA sums of the tile counts of its chunk of sorted pairs
__global__ void __launch_bounds__(kThreads) k_count_sums(const uint64_t *__restrict__ srect,
                                                         int64_t n_total, const uint32_t *n_valid,
                                                         uint32_t *__restrict__ block_sums)
{
    __shared__ unsigned long long s_sum[kWarps];
    const int64_t n = clamp_count(n_valid, n_total);
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b = chunk * blockIdx.x;
    const int64_t e = b + chunk < n ? b + chunk : n;
    unsigned long long sum = 0;
    for (int64_t j = b + threadIdx.x; j < e; j += kThreads) sum += rect_count(srect[j]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kWarps; ++w) t += s_sum[w];
        block_sums[blockIdx.x] = t > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(t);
    }
}

// exclusive scan of the CTA sums (grid <= kScanGrid entries, kScanPer consecutive ones per
// thread); total -> *d_count (saturated)
constexpr int kScanPer = kScanGrid / 1024;
static_assert(kScanGrid % 1024 == 0, "the CTA-sum scan takes whole runs of 1024");
__global__ void __launch_bounds__(1024) k_scan_sums(uint32_t *__restrict__ block_sums, int grid,
                                                    int64_t max_pairs, uint32_t *d_count,
                                                    uint32_t *status)
{
    __shared__ unsigned long long s_w[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t e[kScanPer];
    unsigned long long v = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const int b = tid * kScanPer + i;
        e[i] = b < grid ? block_sums[b] : 0u;
        v += e[i];
    }
    unsigned long long x = v;   // warp inclusive scan, then the warps' totals scanned by warp 0
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = s_w[lane];
        unsigned long long z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, z, o);
            if (lane >= o) z += y;
        }
        s_w[lane] = z - w;
    }
    __syncthreads();
    const unsigned long long incl = x + s_w[warp];
    unsigned long long run = incl - v;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        const int b = tid * kScanPer + i;
        if (b < grid) block_sums[b] = run > 0xFFFFFFFFull ? 0xFFFFFFFFu : static_cast<uint32_t>(run);
        run += e[i];
    }
    if (tid == 1023) {
        const unsigned long long total = incl;
        if (total > static_cast<unsigned long long>(max_pairs)) {
            atomicOr(status, SPLAT_STATUS_CAPACITY);
            *d_count = static_cast<uint32_t>(max_pairs);
        } else {
            *d_count = static_cast<uint32_t>(total);
        }
    }
}

// Emission: each CTA takes its chunk of sorted pairs 256 at a time, reading the pair ids and
// their tile rectangles in sorted order; a CTA scan of the tile counts gives every pair its run
// of output entries, and then each thread writes one entry at a time -- consecutive threads,
// consecutive entries -- finding its pair by binary search over the run ends.  Entry k of a
// pair with tile columns tc0 .. tc0 + ntc - 1 (mod tiles_c) and first tile row tr0 is tile row
// tr0 + k / ntc, column tc0 + k % ntc: row-major over the pair's tile rectangle.
__global__ void __launch_bounds__(kThreads) k_emit(
    const uint32_t *__restrict__ sorted, const uint64_t *__restrict__ srect, int64_t n_total,
    const uint32_t *n_valid, const ViewDesc *__restrict__ views, int64_t n_per_view,
    const uint32_t *__restrict__ block_base, uint32_t *__restrict__ tile_keys,
    uint32_t *__restrict__ tile_vals, int64_t max_pairs)
{
    __shared__ uint32_t s_warp[kWarps];
    __shared__ uint32_t s_carry;
    __shared__ uint32_t s_end[kThreads];    // end of each pair's run inside the batch
    __shared__ uint32_t s_p[kThreads];      // pair id
    __shared__ uint32_t s_row0[kThreads];   // global id of the tile (first tile row, column 0)
    __shared__ int s_tc0[kThreads], s_ntc[kThreads], s_tilesc[kThreads];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = clamp_count(n_valid, n_total);
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b = chunk * blockIdx.x;
    const int64_t e = b + chunk < n ? b + chunk : n;
    const uint32_t npv = static_cast<uint32_t>(n_per_view);
    if (tid == 0) s_carry = block_base[blockIdx.x];
    __syncthreads();
    for (int64_t base = b; base < e; base += kThreads) {
        const int64_t j = base + tid;
        uint32_t p = 0, cnt = 0;
        uint64_t w = 0;
        if (j < e) {
            p = sorted[j];
            w = srect[j];
            cnt = rect_count(w);
        }
        // block inclusive scan of cnt
        uint32_t x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        if (cnt) {
            const ViewDesc &vd = views[p / npv];
            s_row0[tid] = static_cast<uint32_t>(vd.tile_offset +
                                                static_cast<int64_t>(w & 0xFFFFu) * vd.tiles_c);
            s_tc0[tid] = static_cast<int>((w >> 32) & 0xFFFFu);
            s_ntc[tid] = static_cast<int>(w >> 48);
            s_tilesc[tid] = vd.tiles_c;
        }
        s_p[tid] = p;
        __syncthreads();
        uint32_t wbase = 0, total = 0;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) {
            const uint32_t sw = s_warp[k];
            wbase += k < warp ? sw : 0u;
            total += sw;
        }
        s_end[tid] = wbase + x;
        __syncthreads();
        const uint64_t carry = s_carry;
        for (uint32_t q = tid; q < total; q += kThreads) {
            int lo = 0, hi = kThreads - 1;   // first pair whose run ends after q
#pragma unroll
            for (int step = 0; step < 8; ++step) {
                const int mid = (lo + hi) >> 1;
                if (s_end[mid] > q) hi = mid; else lo = mid + 1;
            }
            const uint32_t k = q - (lo ? s_end[lo - 1] : 0u);
            const uint32_t ntc = static_cast<uint32_t>(s_ntc[lo]);
            const uint32_t row = k / ntc;
            int tc = s_tc0[lo] + static_cast<int>(k - row * ntc);
            const int tiles_c = s_tilesc[lo];
            tc = tc >= tiles_c ? tc - tiles_c : tc;
            const uint64_t o = carry + q;
            if (o < static_cast<uint64_t>(max_pairs)) {
                tile_keys[o] = s_row0[lo] + row * static_cast<uint32_t>(tiles_c) +
                               static_cast<uint32_t>(tc);
                tile_vals[o] = s_p[lo];
            }
        }
        __syncthreads();
        if (tid == 0) s_carry += total;
        __syncthreads();
    }
}

// K4: [start, end) per tile from sorted tile ids (ranges zeroed before), and each entry's pixel
// rectangle inside its tile, so that the renderer's warps (eight per tile) need not each gather
// the record and clip it
__global__ void k_ranges(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ vals,
                         const uint64_t *__restrict__ prect, const TileInfo *__restrict__ tiles,
                         int tile_h, int tile_w, const uint32_t *d_count, int64_t max_pairs,
                         uint2 *__restrict__ ranges, uint32_t *__restrict__ entry_rect,
                         uint8_t *__restrict__ entry_blocks)
{
    const int64_t m = clamp_count(d_count, max_pairs);
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < m;
         j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const uint32_t t = keys[j];
        if (j == 0 || keys[j - 1] != t) ranges[t].x = static_cast<uint32_t>(j);
        if (j == m - 1 || keys[j + 1] != t) ranges[t].y = static_cast<uint32_t>(j + 1);
        const TileInfo &ti = tiles[t];
        const uint32_t r = tile_local_rect(unpack_pixel_rect(prect[vals[j]]), ti.tr, ti.tc,
                                           ti.cols, tile_h, tile_w);
        entry_rect[j] = r;
        entry_blocks[j] = static_cast<uint8_t>(rect_blocks(r & ~kRectFlip, tile_h, tile_w));
    }
}

// work order of the compositing kernels: longest lists first, by log2 of the length, so that
// the persistent queue ends on short items (one CTA; a few microseconds)
__global__ void __launch_bounds__(1024) k_order_tiles(const uint2 *__restrict__ ranges,
                                                      int64_t n_tiles, uint32_t *__restrict__ order)
{
    __shared__ uint32_t s_cnt[33], s_off[33];
    const int tid = threadIdx.x;
    if (tid < 33) s_cnt[tid] = 0;
    __syncthreads();
    for (int64_t t = tid; t < n_tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        const uint32_t len = r.y - r.x;
        atomicAdd(&s_cnt[len ? 32 - __clz(len) : 0], 1u);
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t run = 0;
        for (int b = 32; b >= 0; --b) {
            s_off[b] = run;
            run += s_cnt[b];
        }
    }
    __syncthreads();
    for (int64_t t = tid; t < n_tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        const uint32_t len = r.y - r.x;
        order[atomicAdd(&s_off[len ? 32 - __clz(len) : 0], 1u)] = static_cast<uint32_t>(t);
    }
}

}  // namespace

cudaError_t launch_order_tiles(const uint2 *ranges, int64_t n_tiles, uint32_t *order,
                               cudaStream_t st)
{
    if (n_tiles <= 0) return cudaSuccess;
    k_order_tiles<<<1, 1024, 0, st>>>(ranges, n_tiles, order);
    return cudaGetLastError();
}

cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, uint32_t *keys_alt, uint32_t *vals_alt,
                             const uint32_t *d_count, int64_t max_n, int bits, uint32_t *tmp_hist,
                             uint32_t **keys_out, uint32_t **vals_out, cudaStream_t st,
                             const uint32_t *d_count_kept, const uint64_t *aux_in,
                             uint64_t *aux_out)
{
    uint32_t *kin = keys, *vin = vals, *kout = keys_alt, *vout = vals_alt;
    if (max_n > 0) {
        for (int shift = 0; shift < bits; shift += 8) {
            uint32_t *dtot = tmp_hist + kSortGrid * kRadix;
            // with d_count_kept, the first pass drops the key 0xFFFFFFFF and the later passes
            // sort the d_count_kept items left
            const int drop = d_count_kept && shift == 0;
            const uint32_t *cnt = d_count_kept && shift > 0 ? d_count_kept : d_count;
            k_upsweep<<<kSortGrid, kThreads, 0, st>>>(kin, cnt, max_n, shift, drop, tmp_hist);
            k_scan_digits<<<kRadix / 8, 256, 0, st>>>(tmp_hist, kSortGrid, dtot);
            const bool last = shift + 8 >= bits;
            k_downsweep<<<kSortGrid, kThreads, 0, st>>>(kin, vin, kout, vout, cnt, max_n, shift,
                                                        drop, tmp_hist, dtot, aux_in,
                                                        last ? aux_out : nullptr);
            uint32_t *t = kin;
            kin = kout;
            kout = t;
            t = vin;
            vin = vout;
            vout = t;
        }
    }
    *keys_out = kin;
    *vals_out = vin;
    return cudaGetLastError();
}

cudaError_t launch_emit(const uint32_t *sorted_pair_ids, const uint64_t *sorted_trect,
                        int64_t n_pairs_total, const uint32_t *n_valid, const ViewDesc *views,
                        int64_t n_per_view, uint32_t *block_sums, uint32_t *tile_keys,
                        uint32_t *tile_vals, int64_t max_pairs, uint32_t *d_count,
                        uint32_t *status, cudaStream_t st)
{
    k_count_sums<<<kScanGrid, kThreads, 0, st>>>(sorted_trect, n_pairs_total, n_valid, block_sums);
    k_scan_sums<<<1, 1024, 0, st>>>(block_sums, kScanGrid, max_pairs, d_count, status);
    k_emit<<<kScanGrid, kThreads, 0, st>>>(sorted_pair_ids, sorted_trect, n_pairs_total, n_valid,
                                           views, n_per_view, block_sums, tile_keys, tile_vals,
                                           max_pairs);
    return cudaGetLastError();
}

cudaError_t launch_ranges(const uint32_t *tile_keys, const uint32_t *tile_vals,
                          const uint64_t *prect, const TileInfo *tiles, int tile_h, int tile_w,
                          const uint32_t *d_count, int64_t max_pairs, uint2 *ranges,
                          int64_t n_tiles, uint32_t *entry_rect, uint8_t *entry_blocks,
                          cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * static_cast<size_t>(n_tiles), st);
    if (e != cudaSuccess) return e;
    k_ranges<<<kRangesGrid, 256, 0, st>>>(tile_keys, tile_vals, prect, tiles, tile_h, tile_w,
                                            d_count, max_pairs, ranges, entry_rect,
                                            entry_blocks);
    return cudaGetLastError();
}

}  // namespace splat
