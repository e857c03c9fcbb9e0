// gs_sort.cu -- A2-A4 binning: deterministic (tile, depth, index) order.
//
// The order the rasteriser needs (paper Sec. II: depth sorting; Sec. III-B:
// tile-based rasterisation) is that of the key (tile, depth, view*n+index).
// It is produced as one stable LSD radix sort whose low digits -- the 32 bits
// of the FP32 depth -- are sorted once per (view, Gaussian) *before* the
// instances are emitted (all instances of a Gaussian share its depth), and
// whose high digits -- the global tile id -- are sorted over the emitted
// instances.  Emission walks the depth order, so the instance array enters
// the tile passes already in (depth, view, index) order and stability keeps
// it.  Per pass: a per-block digit histogram, a per-digit scan over blocks and
// a stable block-local ranking with warp match + per-warp counters, scattered
// to the digit's global offset.  The first depth pass drops the (view,
// Gaussian) pairs the projection culled (key 0xFFFFFFFF, no tile): the later
// passes, the scan and the emission run over the visible pairs only, whose
// count stays on the device like the instance count.  No kernel waits on
// another block, so nothing can spin.
#include <atomic>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kWarps = kSortThreads / 32;
constexpr int kGridPerSm = 8;  // CTAs per SM of the grid-stride kernels
constexpr uint32_t kCulledKey = 0xFFFFFFFFu;  // depth key of a culled pair (never a depth)

__device__ __forceinline__ uint32_t active_count(const uint32_t* count_dev, uint32_t count_host) {
    return count_dev ? *count_dev : count_host;
}

// Block-wide exclusive scan of one value per thread (kSortThreads threads).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* warp_tot,
                                                         uint32_t& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = ti - t;
        if (lane == (int)(blockDim.x >> 5) - 1) warp_tot[32] = ti;
    }
    __syncthreads();
    uint32_t r = inc - x + warp_tot[w];
    total = warp_tot[32];
    __syncthreads();
    return r;
}

// Radix passes over blocks of ITEMS keys per thread (TILE = 256 * ITEMS keys
// per block).
template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads)
k_radix_hist(const uint32_t* __restrict__ keys, const uint32_t* count_dev, uint32_t count_host,
             uint32_t cap, int shift, uint32_t mask, int nb, int drop,
             uint32_t* __restrict__ hist) {
    grid_dep_begin();
    constexpr int TILE = kSortThreads * ITEMS;
    __shared__ uint32_t h[kRadix];
    const uint32_t count = min(active_count(count_dev, count_host), cap);
    // a grid of resident CTAs striding over the sort blocks of the active keys
    for (uint32_t blk = blockIdx.x; blk * (uint32_t)TILE < count; blk += gridDim.x) {
        const uint32_t start = blk * (uint32_t)TILE;
        h[threadIdx.x] = 0u;
        __syncthreads();
        const uint32_t end = min(start + (uint32_t)TILE, count);
        for (uint32_t i = start + threadIdx.x; i < end; i += kSortThreads) {
            const uint32_t k = keys[i];
            if (!(drop && k == kCulledKey)) atomicAdd(&h[(k >> shift) & mask], 1u);
        }
        __syncthreads();
        hist[(size_t)threadIdx.x * nb + blk] = h[threadIdx.x];
    }
}

// One block per digit: exclusive scan of the digit's per-block counts (in
// place) and the digit total.
template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads)
k_radix_scan(uint32_t* __restrict__ hist, const uint32_t* count_dev, uint32_t count_host,
             uint32_t cap, int nb, uint32_t* __restrict__ totals) {
    grid_dep_begin();
    constexpr int TILE = kSortThreads * ITEMS;
    __shared__ uint32_t wt[33];
    const uint32_t count = min(active_count(count_dev, count_host), cap);
    const int active = (int)((count + TILE - 1) / TILE);
    uint32_t* row = hist + (size_t)blockIdx.x * nb;
    uint32_t carry = 0;
    for (int base = 0; base < active; base += kSortThreads * 4) {
        uint32_t v[4], s = 0;
        for (int k = 0; k < 4; ++k) {
            int i = base + threadIdx.x * 4 + k;
            v[k] = i < active ? row[i] : 0u;
            s += v[k];
        }
        uint32_t tot;
        uint32_t ex = block_exclusive_scan(s, wt, tot);
        uint32_t run = carry + ex;
        for (int k = 0; k < 4; ++k) {
            int i = base + threadIdx.x * 4 + k;
            if (i < active) row[i] = run;
            run += v[k];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

// Stable scatter of one block of keys: each key's rank among the block's keys
// of its digit comes from per-warp match_any ranking; the block is first
// reordered by digit in shared memory, so the global writes of each digit's
// run are consecutive addresses (coalesced) instead of one scattered word per
// key.  With drop, culled keys are neither ranked nor written, and block 0
// stores the number of keys the pass keeps in *kept_out.  Without vals_in
// the value of key i is i.
template <int ITEMS>
__global__ void __launch_bounds__(kSortThreads)
k_radix_scatter(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                const uint32_t* count_dev, uint32_t count_host, uint32_t cap, int shift,
                uint32_t mask, int nb,
                const uint32_t* __restrict__ hist, const uint32_t* __restrict__ totals, int drop,
                uint32_t* __restrict__ kept_out) {
    grid_dep_begin();
    constexpr int TILE = kSortThreads * ITEMS;
    constexpr int kWarpItems = TILE / kWarps;  // consecutive keys per warp
    __shared__ uint32_t base[kRadix];          // global start of the digit's run of this block
    __shared__ uint32_t local[kRadix];         // start of the digit's run inside the block
    __shared__ uint32_t wcnt[kWarps][kRadix];
    __shared__ uint32_t wt[33];
    __shared__ uint32_t skey[TILE], sval[TILE];
    const uint32_t count = min(active_count(count_dev, count_host), cap);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // a grid of resident CTAs striding over the sort blocks of the active keys
    for (uint32_t blk = blockIdx.x; blk * (uint32_t)TILE < count; blk += gridDim.x) {
        const uint32_t start = blk * (uint32_t)TILE;
        // the block's keys and values are loaded first, so that their latency
        // overlaps the loads and the scan of the digit offsets below
        uint32_t key[ITEMS], val[ITEMS], rank[ITEMS];
        const uint32_t wstart = start + (uint32_t)w * kWarpItems;
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const uint32_t i = wstart + (uint32_t)r * 32u + lane;
            const bool in = i < count;
            key[r] = in ? keys_in[i] : 0u;
            val[r] = in ? (vals_in ? vals_in[i] : i) : 0u;
        }
        {
            uint32_t tot;
            uint32_t ex = block_exclusive_scan(totals[tid], wt, tot);
            base[tid] = ex + hist[(size_t)tid * nb + blk];
            if (kept_out && blk == 0 && tid == 0) *kept_out = tot;  // keys of all digits
        }
#pragma unroll
        for (int k = 0; k < kWarps; ++k) wcnt[k][tid] = 0u;
        __syncthreads();

        const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const uint32_t i = wstart + (uint32_t)r * 32u + lane;
            const bool in = i < count;
            const bool ok = in && !(drop && key[r] == kCulledKey);
            const uint32_t d = ok ? ((key[r] >> shift) & mask) : 0x10000u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            uint32_t rk = 0u;
            if (ok) rk = wcnt[w][d] + __popc(peers & lt);
            __syncwarp();
            if (ok && (__ffs(peers) - 1) == lane) wcnt[w][d] += __popc(peers);
            __syncwarp();
            rank[r] = rk;
        }
        __syncthreads();
        uint32_t digit_count = 0u;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) {
            const uint32_t c = wcnt[k][tid];
            wcnt[k][tid] = digit_count;
            digit_count += c;
        }
        uint32_t n_kept;  // keys of this block that are written (all of them without drop)
        local[tid] = block_exclusive_scan(digit_count, wt, n_kept);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const uint32_t i = wstart + (uint32_t)r * 32u + lane;
            if (i < count && !(drop && key[r] == kCulledKey)) {
                const uint32_t d = (key[r] >> shift) & mask;
                const uint32_t s = local[d] + wcnt[w][d] + rank[r];
                skey[s] = key[r];
                sval[s] = val[r];
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const int s = r * kSortThreads + tid;
            if ((uint32_t)s < n_kept) {
                const uint32_t k = skey[s];
                const uint32_t d = (k >> shift) & mask;
                const uint32_t pos = base[d] + ((uint32_t)s - local[d]);
                keys_out[pos] = k;
                vals_out[pos] = sval[s];
            }
        }
        __syncthreads();  // the next block reuses the shared arrays
    }
}

// Sum of tiles touched over each scan block, in depth order (the first
// *count_dev entries of order: the visible pairs).
__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t* __restrict__ order, const uint32_t* __restrict__ touched,
              const uint32_t* count_dev, uint32_t* __restrict__ block_sums) {
    grid_dep_begin();
    __shared__ uint32_t wt[33];
    const uint32_t count = *count_dev;
    const uint32_t start = blockIdx.x * (uint32_t)kScanTile;
    uint32_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t i = start + threadIdx.x * kScanItems + k;
        if (i < count) s += touched[order[i]];
    }
    uint32_t tot;
    block_exclusive_scan(s, wt, tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Sum over the CTA of one 64-bit value per thread (kScanThreads threads);
// valid in every thread.
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long x,
                                                          unsigned long long* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[w] = x;
    __syncthreads();
    unsigned long long t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    __syncthreads();
    return t;
}

// Global exclusive offsets of the instances of every visible (view,
// Gaussian) entry in depth order: off[i] for i < count, off[count] = total
// (count = *count_dev).  Each CTA forms its own starting offset from the
// block sums before it (a few hundred words), so no separate scan of the
// block sums runs; CTA 0 also forms the total and the instance counters
// (vn = the number of depth-order entries, for later readers).
__global__ void __launch_bounds__(kScanThreads)
k_scan_offsets(const uint32_t* __restrict__ order, const uint32_t* __restrict__ touched,
               const uint32_t* __restrict__ block_sums, int nb, uint32_t cap,
               const uint32_t* count_dev, DevCounters* ctr, uint32_t* __restrict__ off) {
    grid_dep_begin();
    __shared__ uint32_t wt[33];
    __shared__ unsigned long long red[kScanThreads / 32];
    const uint32_t count = *count_dev;
    unsigned long long pre = 0;
    for (int i = threadIdx.x; i < (int)blockIdx.x; i += blockDim.x) pre += block_sums[i];
    pre = block_sum_u64(pre, red);
    if (blockIdx.x == 0) {
        unsigned long long tot = 0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) tot += block_sums[i];
        tot = block_sum_u64(tot, red);
        if (threadIdx.x == 0) {
            ctr->n_raw = tot;
            ctr->vn = count;
            ctr->n_instances = (uint32_t)min(tot, (unsigned long long)cap);
            if (tot > cap) atomicOr(&ctr->status, (uint32_t)GS_DEV_CAPACITY);
        }
    }
    const uint32_t start = blockIdx.x * (uint32_t)kScanTile;
    uint32_t t[kScanItems], s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t i = start + threadIdx.x * kScanItems + k;
        t[k] = i < count ? touched[order[i]] : 0u;
        s += t[k];
    }
    uint32_t tot;
    uint32_t o = block_exclusive_scan(s, wt, tot) +
                 (uint32_t)min(pre, (unsigned long long)0xFFFFFFFFu);
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t i = start + threadIdx.x * kScanItems + k;
        if (i < count) {
            off[i] = o;
            if (i + 1 == count) off[count] = o + t[k];  // the total
        }
        o += t[k];
    }
}

// Emit one instance per (Gaussian, tile in its rect), walking the depth
// order; tiles of a rect in row-major order.  Each CTA takes kEmitEntries
// consecutive entries and writes their instances consecutively, in rounds
// of kEmitRun * kEmitEntries output slots: every thread fills a run of
// kEmitRun consecutive slots (one binary search over the entries' offsets in
// shared memory for the run's first slot, then tile after tile of the entry
// and on to the next entry) into a shared-memory copy of the round, which the
// CTA then writes out with coalesced stores.  No thread is left alone with a
// large rect.
constexpr int kEmitEntries = 256;
constexpr int kEmitRun = 8;
constexpr int kEmitRound = kEmitRun * kEmitEntries;
// shared-memory slot of round position q: one pad word per 32, so that the
// runs' writes (stride kEmitRun) and the write-out's reads (stride 1) are free
// of bank conflicts
__device__ __forceinline__ int emit_slot(int q) { return q + (q >> 5); }

__global__ void __launch_bounds__(kEmitEntries)
k_emit(const uint32_t* __restrict__ order, const uint32_t* __restrict__ off,
       const uint2* __restrict__ rects, const uint32_t* count_dev, int n, ViewTable vt,
       uint32_t cap,
       uint32_t* __restrict__ ikeys, uint32_t* __restrict__ ivals,
       uint32_t* __restrict__ gid_of, const uint32_t* __restrict__ spans,
       const uint32_t* __restrict__ pool) {
    grid_dep_begin();
    __shared__ uint32_t s_off[kEmitEntries + 1];
    __shared__ uint32_t s_vg[kEmitEntries];
    __shared__ uint2 s_rect[kEmitEntries];
    // tight rects: the entry's row spans (boxes of at most kSpanRows rows),
    // or, for a taller box, the pool index of its first row in s_span[e][0]
    __shared__ __align__(16) uint32_t s_span[kEmitEntries][kSpanRows];
    __shared__ uint16_t s_view[kEmitEntries];
    // the round's instances: tile keys and (view, Gaussian) indices
    __shared__ uint32_t s_key[kEmitRound + kEmitRound / 32];
    __shared__ uint32_t s_val[kEmitRound + kEmitRound / 32];
    const uint32_t count = *count_dev;
    // a grid of resident CTAs striding over the groups of entries
    for (uint32_t e0 = blockIdx.x * (uint32_t)kEmitEntries; e0 < count;
         e0 += gridDim.x * (uint32_t)kEmitEntries) {
        const uint32_t ne = min((uint32_t)kEmitEntries, count - e0);
        const int e = threadIdx.x;
        if ((uint32_t)e < ne) {
            const uint32_t vg = order[e0 + e];
            const uint32_t o0 = off[e0 + e], o1 = off[e0 + e + 1];
            const uint2 rc = rects[vg];
            // whole 16-byte groups of the entry's 64-byte span record; the
            // first (rows 0-3) is loaded beside the rect, the others only for
            // taller boxes
            const uint4* src = reinterpret_cast<const uint4*>(spans + (size_t)vg * kSpanRows);
            const uint4 sp0 = vt.tight_rect ? src[0] : make_uint4(0u, 0u, 0u, 0u);
            s_off[e] = o0;
            s_vg[e] = vg;
            s_rect[e] = rc;
            s_view[e] = (uint16_t)(vg / (uint32_t)n);
            if (vt.tight_rect && o0 != o1) {
                const int rows = (int)(rc.y >> 16) - (int)(rc.x >> 16);
                const int nw = rows > kSpanRows ? 1 : rows;
                uint4* dst = reinterpret_cast<uint4*>(s_span[e]);
                dst[0] = sp0;
                for (int q = 1; q < (nw + 3) / 4; ++q) dst[q] = src[q];
            }
        }
        if (e == 0) s_off[ne] = off[e0 + ne];
        __syncthreads();
        const uint32_t first = s_off[0], stop = min(s_off[ne], cap);
        for (uint32_t base = first; base < stop; base += kEmitRound) {
            const uint32_t nr = min((uint32_t)kEmitRound, stop - base);  // slots of this round
            uint32_t p = base + (uint32_t)threadIdx.x * kEmitRun;
            const uint32_t p_end = min(p + kEmitRun, base + nr);
            if (p < p_end) {
                int lo = 0, hi = (int)ne;  // invariant: s_off[lo] <= p < s_off[hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (s_off[mid] <= p) lo = mid; else hi = mid;
                }
                for (;;) {
                    // entry lo's tiles k = p - s_off[lo], ... of this run
                    const uint32_t e_end = min(s_off[lo + 1], p_end);
                    const uint2 rc = s_rect[lo];
                    const uint32_t x0 = rc.x & 0xFFFF, y0 = rc.x >> 16, x1 = rc.y & 0xFFFF,
                                   y1 = rc.y >> 16;
                    const ViewGeom& geo = vt.v[s_view[lo]];
                    const uint32_t kbase = (uint32_t)geo.tile_offset, tiles_x = (uint32_t)geo.tiles_x;
                    const uint32_t vg = s_vg[lo];
                    const uint32_t k = p - s_off[lo];
                    const bool tall = y1 - y0 > (uint32_t)kSpanRows;
                    if (vt.tight_rect && !(tall && s_span[lo][0] == kSpanNoPool)) {
                        // the k-th tile of the row spans the projection stored and
                        // counted, then the ones after it (row r, kk-th tile of the row)
                        const uint32_t* sr = tall ? pool + s_span[lo][0] : s_span[lo];
                        const uint32_t nrows = y1 - y0;
                        uint32_t kk = k, r = 0, sp = sr[0];
                        for (;;) {
                            for (; r + 1 < nrows; ++r) {
                                const uint32_t wr = (sp >> 16) - (sp & 0xFFFF);
                                if (kk < wr) break;
                                kk -= wr;
                                sp = sr[r + 1];
                            }
                            // (a count that disagreed would land past the row; stay
                            // inside the rect)
                            const uint32_t tx = min((sp & 0xFFFF) + kk, x1 - 1u);
                            const int q = emit_slot((int)(p - base));
                            s_key[q] = kbase + (y0 + r) * tiles_x + tx;
                            s_val[q] = vg;
                            if (++p == e_end) break;
                            ++kk;
                        }
                    } else {
                        const uint32_t w = x1 - x0;
                        const uint32_t dy = k / w;
                        uint32_t ty = y0 + dy, tx = x0 + (k - dy * w);
                        for (;;) {
                            const int q = emit_slot((int)(p - base));
                            s_key[q] = kbase + ty * tiles_x + tx;
                            s_val[q] = vg;
                            if (++p == e_end) break;
                            if (++tx == x1) {
                                tx = x0;
                                ++ty;
                            }
                        }
                    }
                    if (p == p_end) break;
                    // the next entry with instances
                    do {
                        ++lo;
                    } while (s_off[lo + 1] <= p);
                }
            }
            __syncthreads();
            for (uint32_t q = threadIdx.x; q < nr; q += kEmitEntries) {
                const uint32_t pos = base + q;
                const int sq = emit_slot((int)q);
                ikeys[pos] = s_key[sq];
                if (gid_of) {
                    // deterministic plans: the sort carries the emission position
                    ivals[pos] = pos;
                    gid_of[pos] = s_val[sq];
                } else {
                    ivals[pos] = s_val[sq];
                }
            }
            __syncthreads();
        }
        __syncthreads();  // the next group reuses the shared arrays
    }
}

// Per-tile [begin, end) of the sorted instance keys: a tile's range starts
// where the key differs from the one before it and ends where it differs from
// the one after.  Each thread takes four consecutive keys (one 16-byte load;
// the workspace's buffers are 256-byte aligned) and the keys on either side.
__global__ void k_ranges(const uint32_t* __restrict__ keys, const uint32_t* count_dev,
                         uint32_t* __restrict__ ranges, uint32_t* __restrict__ order_scratch) {
    grid_dep_begin();
    // the tile order's bucket counts and cursors start at zero
    if (blockIdx.x == 0 && threadIdx.x < 2 * kOrderBuckets) order_scratch[threadIdx.x] = 0u;
    constexpr uint32_t kNone = 0xFFFFFFFFu;  // past either end (never a tile id)
    const uint32_t count = *count_dev;
    const uint32_t ngroups = (count + 3) / 4;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups;
         g += gridDim.x * blockDim.x) {
        const uint32_t i0 = 4 * g;
        uint32_t k[6];  // the keys at i0 - 1 .. i0 + 4
        if (i0 + 4 <= count) {
            const uint4 v = reinterpret_cast<const uint4*>(keys)[g];
            k[1] = v.x;
            k[2] = v.y;
            k[3] = v.z;
            k[4] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) k[1 + j] = i0 + j < count ? keys[i0 + j] : kNone;
        }
        k[0] = i0 > 0 ? keys[i0 - 1] : kNone;
        k[5] = i0 + 4 < count ? keys[i0 + 4] : kNone;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t key = k[1 + j];
            if (key == kNone) break;
            if (k[j] != key) ranges[2 * key] = i0 + j;
            if (k[2 + j] != key) ranges[2 * key + 1] = i0 + j + 1;
        }
    }
}

// Heavy-first order of the tiles for the render kernels: tiles bucketed by
// the bit length of their list length, longest bucket first, so the CTAs of
// the longest lists start in the first wave instead of forming the tail.
// Two grid-wide passes: the bucket sizes (per-CTA counts added to global
// counters), then each tile's slot (the bucket's start plus a cursor taken
// with one atomic per warp and bucket).  Within a bucket the order is
// arbitrary: it changes scheduling, never a result.
constexpr int kOrderThreads = 256;

__device__ __forceinline__ int work_bucket(const uint32_t* ranges, int t) {
    const uint32_t len = ranges[2 * t + 1] - ranges[2 * t];
    return len == 0u ? kOrderBuckets - 1 : __clz(len);  // 0 = longest
}

__global__ void __launch_bounds__(kOrderThreads)
k_tile_buckets(const uint32_t* __restrict__ ranges, int T, uint32_t* __restrict__ counts) {
    grid_dep_begin();
    __shared__ uint32_t cnt[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) cnt[threadIdx.x] = 0u;
    __syncthreads();
    for (int t = blockIdx.x * kOrderThreads + threadIdx.x; t < T; t += gridDim.x * kOrderThreads)
        atomicAdd(&cnt[work_bucket(ranges, t)], 1u);
    __syncthreads();
    if (threadIdx.x < kOrderBuckets && cnt[threadIdx.x] != 0u)
        atomicAdd(&counts[threadIdx.x], cnt[threadIdx.x]);
}

__global__ void __launch_bounds__(kOrderThreads)
k_tile_order(const uint32_t* __restrict__ ranges, int T, const uint32_t* __restrict__ counts,
             uint32_t* __restrict__ cursors, uint32_t* __restrict__ order) {
    grid_dep_begin();
    __shared__ uint32_t base[kOrderBuckets];
    if (threadIdx.x == 0) {
        uint32_t run = 0u;
        for (int b = 0; b < kOrderBuckets; ++b) {
            base[b] = run;
            run += counts[b];
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    for (int t0 = blockIdx.x * kOrderThreads; t0 < T; t0 += gridDim.x * kOrderThreads) {
        const int t = t0 + threadIdx.x;
        const int b = t < T ? work_bucket(ranges, t) : 1000 + lane;  // unique dummy
        const uint32_t peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1;
        uint32_t first = 0u;
        if (t < T && leader == lane) first = atomicAdd(&cursors[b], __popc(peers));
        first = __shfl_sync(0xffffffffu, first, leader);
        if (t < T) order[base[b] + first + __popc(peers & lt)] = (uint32_t)t;
    }
}

// CTAs of a grid-stride kernel resident at once on this GPU (its occupancy
// per SM, cached per kernel, times the SMs): the binning's kernels whose work
// is counted on the device launch this many at most, so that no CTA is
// launched only to find nothing to do.
template <auto Kernel>
int resident_grid(int threads) {
    static std::atomic<int> per_sm{0};
    int b = per_sm.load(std::memory_order_relaxed);
    if (b <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, Kernel, threads, 0) !=
                cudaSuccess ||
            b < 1)
            b = 1;
        per_sm.store(b, std::memory_order_relaxed);
    }
    return b * sm_count();
}

template <int ITEMS>
gs_status radix_pass_t(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout,
                       const uint32_t* count_dev, uint32_t count_host, uint32_t cap, int shift,
                       int bits, uint32_t* hist, uint32_t* totals, uint32_t* kept_out,
                       cudaStream_t st) {
    const int nb = (int)((cap + kSortThreads * ITEMS - 1) / (kSortThreads * ITEMS));
    const int drop = kept_out != nullptr;
    const uint32_t mask = (1u << bits) - 1u;
    const int hg = min(nb, resident_grid<k_radix_hist<ITEMS>>(kSortThreads));
    const int sg = min(nb, resident_grid<k_radix_scatter<ITEMS>>(kSortThreads));
    launch_pdl(k_radix_hist<ITEMS>, hg, kSortThreads, 0, st, kin, count_dev, count_host, cap,
               shift, mask, nb, drop, hist);
    launch_pdl(k_radix_scan<ITEMS>, kRadix, kSortThreads, 0, st, hist, count_dev, count_host,
               cap, nb, totals);
    launch_pdl(k_radix_scatter<ITEMS>, sg, kSortThreads, 0, st, kin, vin, kout, vout, count_dev,
               count_host, cap, shift, mask, nb, hist, totals, drop, kept_out);
    return launch_status();
}

// One stable pass on `bits` (<= 8) bits at `shift` over up to `cap` keys (the real count
// comes from count_dev when given), in blocks of 1024 keys: measured faster
// than blocks of 2048 or 4096 for both the 1M depth keys and the 5M instances
// (with the digit-reordered, coalesced writes too).  With kept_out the pass
// drops the culled keys and stores how many it kept there.
template <int ITEMS = kSortItems>
gs_status radix_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout,
                     const uint32_t* count_dev, uint32_t count_host, uint32_t cap, int shift,
                     int bits, uint32_t* hist, uint32_t* totals, cudaStream_t st,
                     uint32_t* kept_out = nullptr) {
    static_assert(ITEMS >= kSortItems, "the histogram buffer holds kSortTile-key blocks");
    return radix_pass_t<ITEMS>(kin, vin, kout, vout, count_dev, count_host, cap, shift, bits,
                               hist, totals, kept_out, st);
}

}  // namespace

gs_status launch_bin_sort(const Plan* p, int32_t n, void* ws, cudaStream_t st) {
    const uint32_t VN = (uint32_t)p->vt.n_views * (uint32_t)n;
    const uint32_t icap = (uint32_t)p->inst_capacity;
    uint32_t* hist = buf<uint32_t>(p, ws, B_HIST);
    uint32_t* totals = hist + (size_t)kRadix * (p->depth_sort_blocks > p->inst_sort_blocks
                                                    ? p->depth_sort_blocks
                                                    : p->inst_sort_blocks);
    DevCounters* ctr = buf<DevCounters>(p, ws, GS_BUF_COUNTERS);
    // the per-tile ranges are cleared first, so that every kernel of the
    // binning follows another kernel (programmatic launches, see launch_pdl)
    uint32_t* ranges = buf<uint32_t>(p, ws, GS_BUF_RANGES);
    if (cudaMemsetAsync(ranges, 0, (size_t)p->total_tiles * 2 * sizeof(uint32_t), st) !=
        cudaSuccess)
        return GS_ERR_CUDA;

    // 1. depth digits over the (view, Gaussian) pairs: 4 passes, the
    //    projection's keys (values = positions) -> B -> C -> B -> C; the first
    //    keeps only the visible pairs, whose count (n_sorted) the later passes
    //    read on the device.  The projection's keys are left intact, so a
    //    second binning of the same projection sorts the same pairs.
    const uint32_t* kp = buf<uint32_t>(p, ws, B_DKEY_A);
    uint32_t* kb = buf<uint32_t>(p, ws, B_DKEY_B);
    uint32_t* vb = buf<uint32_t>(p, ws, B_DVAL_B);
    uint32_t* kc = buf<uint32_t>(p, ws, B_DKEY_C);
    uint32_t* va = buf<uint32_t>(p, ws, GS_BUF_DEPTH_ORDER);
    uint32_t* n_sorted = &ctr->n_sorted;
    gs_status s0 = radix_pass(kp, nullptr, kb, vb, nullptr, VN, VN, 0, kRadixBits, hist, totals,
                              st, n_sorted);
    if (s0 != GS_OK) return s0;
    for (int pass = 1; pass < 4; ++pass) {
        const bool odd = (pass & 1) != 0;
        gs_status s = radix_pass(odd ? kb : kc, odd ? vb : va, odd ? kc : kb, odd ? va : vb,
                                 n_sorted, VN, VN, pass * kRadixBits, kRadixBits, hist, totals,
                                 st);
        if (s != GS_OK) return s;
    }

    // 2. scan of tiles touched in depth order, then emission (grids over all
    //    pairs; blocks past the visible count do nothing)
    const int snb = (int)((VN + kScanTile - 1) / kScanTile);
    uint32_t* bsums = buf<uint32_t>(p, ws, B_SCAN_BLOCKS);
    const uint32_t* touched = buf<uint32_t>(p, ws, GS_BUF_TOUCHED);
    launch_pdl(k_scan_reduce, snb, kScanThreads, 0, st, va, touched, n_sorted, bsums);
    uint32_t* ika = buf<uint32_t>(p, ws, GS_BUF_TILE_KEYS);
    uint32_t* iva = buf<uint32_t>(p, ws, GS_BUF_TILE_VALUES);
    uint32_t* ikb = buf<uint32_t>(p, ws, B_IKEY_B);
    uint32_t* ivb = buf<uint32_t>(p, ws, B_IVAL_B);
    uint32_t* offs = buf<uint32_t>(p, ws, B_OFFSETS);
    launch_pdl(k_scan_offsets, snb, kScanThreads, 0, st, va, touched, bsums, snb, icap, n_sorted,
               ctr, offs);
    const int eg = (int)min((VN + kEmitEntries - 1) / kEmitEntries,
                            (uint32_t)resident_grid<k_emit>(kEmitEntries));
    launch_pdl(k_emit, eg, kEmitEntries, 0, st, va, offs,
               buf<uint2>(p, ws, GS_BUF_RECT), n_sorted, n, p->vt, icap, ika, iva,
               p->cfg.deterministic ? buf<uint32_t>(p, ws, B_GID_OF) : nullptr,
               buf<uint32_t>(p, ws, B_SPANS), cbuf<uint32_t>(p, ws, B_SPAN_POOL));
    gs_status s = launch_status();
    if (s != GS_OK) return s;

    // 3. tile-id digits over the instances, the id's bits split evenly over
    //    the passes (14 bits: 7 + 7 rather than 8 + 6, so that both passes
    //    write runs of similar length)
    const uint32_t* cnt = &ctr->n_instances;
    const int tbits = (p->tile_bits + p->tile_passes - 1) / p->tile_passes;
    for (int pass = 0; pass < p->tile_passes; ++pass) {
        const bool even = (pass & 1) == 0;
        s = radix_pass(even ? ika : ikb, even ? iva : ivb, even ? ikb : ika, even ? ivb : iva, cnt,
                       0u, icap, pass * tbits, tbits, hist, totals, st);
        if (s != GS_OK) return s;
    }
    const uint32_t* sorted_keys = (p->tile_passes & 1) ? ikb : ika;

    // 4. per-tile ranges (cleared above)
    const int sms = sm_count();
    if (sms <= 0) return GS_ERR_CUDA;
    uint32_t* order = buf<uint32_t>(p, ws, B_TILE_ORDER);
    uint32_t* order_scratch = order + p->total_tiles;  // bucket counts | cursors
    launch_pdl(k_ranges, sms * kGridPerSm, 256, 0, st, sorted_keys, cnt, ranges, order_scratch);
    int ob = (p->total_tiles + kOrderThreads - 1) / kOrderThreads;
    ob = ob < 4 * sms ? ob : 4 * sms;
    launch_pdl(k_tile_buckets, ob, kOrderThreads, 0, st, ranges, p->total_tiles, order_scratch);
    launch_pdl(k_tile_order, ob, kOrderThreads, 0, st, ranges, p->total_tiles, order_scratch,
               order_scratch + kOrderBuckets, order);
    return launch_status();
}

}  // namespace gs
