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
// to the digit's global offset.  No kernel waits on another block, so nothing
// can spin; the instance count never leaves the device.
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kWarps = kSortThreads / 32;
constexpr int kWarpItems = kSortTile / kWarps;  // 512 consecutive elements per warp
constexpr int kGrid = 152 * 8;                  // grid-stride kernels

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

__global__ void __launch_bounds__(kSortThreads)
k_radix_hist(const uint32_t* __restrict__ keys, const uint32_t* count_dev, uint32_t count_host,
             uint32_t cap, int shift, int nb, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kRadix];
    const uint32_t count = min(active_count(count_dev, count_host), cap);
    const uint32_t start = blockIdx.x * (uint32_t)kSortTile;
    if (start >= count) return;
    h[threadIdx.x] = 0u;
    __syncthreads();
    const uint32_t end = min(start + (uint32_t)kSortTile, count);
    for (uint32_t i = start + threadIdx.x; i < end; i += kSortThreads)
        atomicAdd(&h[(keys[i] >> shift) & (kRadix - 1)], 1u);
    __syncthreads();
    hist[(size_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// One block per digit: exclusive scan of the digit's per-block counts (in
// place) and the digit total.
__global__ void __launch_bounds__(kSortThreads)
k_radix_scan(uint32_t* __restrict__ hist, const uint32_t* count_dev, uint32_t count_host,
             uint32_t cap, int nb, uint32_t* __restrict__ totals) {
    __shared__ uint32_t wt[33];
    const uint32_t count = min(active_count(count_dev, count_host), cap);
    const int active = (int)((count + kSortTile - 1) / kSortTile);
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

__global__ void __launch_bounds__(kSortThreads)
k_radix_scatter(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                const uint32_t* count_dev, uint32_t count_host, uint32_t cap, int shift, int nb,
                const uint32_t* __restrict__ hist, const uint32_t* __restrict__ totals) {
    __shared__ uint32_t base[kRadix];
    __shared__ uint32_t wcnt[kWarps][kRadix];
    __shared__ uint32_t wt[33];
    const uint32_t count = min(active_count(count_dev, count_host), cap);
    const uint32_t start = blockIdx.x * (uint32_t)kSortTile;
    if (start >= count) return;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    {
        uint32_t tot;
        uint32_t ex = block_exclusive_scan(totals[tid], wt, tot);
        base[tid] = ex + hist[(size_t)tid * nb + blockIdx.x];
    }
#pragma unroll
    for (int k = 0; k < kWarps; ++k) wcnt[k][tid] = 0u;
    __syncthreads();

    uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t wstart = start + (uint32_t)w * kWarpItems;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = wstart + (uint32_t)r * 32u + lane;
        const bool ok = i < count;
        key[r] = ok ? keys_in[i] : 0u;
        val[r] = ok ? vals_in[i] : 0u;
        const uint32_t d = ok ? ((key[r] >> shift) & (kRadix - 1)) : 0x10000u;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rk = 0u;
        if (ok) rk = wcnt[w][d] + __popc(peers & lt);
        __syncwarp();
        if (ok && (__ffs(peers) - 1) == lane) wcnt[w][d] += __popc(peers);
        __syncwarp();
        rank[r] = rk;
    }
    __syncthreads();
    {
        uint32_t run = 0u;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) {
            uint32_t c = wcnt[k][tid];
            wcnt[k][tid] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t i = wstart + (uint32_t)r * 32u + lane;
        if (i < count) {
            const uint32_t d = (key[r] >> shift) & (kRadix - 1);
            const uint32_t pos = base[d] + wcnt[w][d] + rank[r];
            keys_out[pos] = key[r];
            vals_out[pos] = val[r];
        }
    }
}

// Sum of tiles touched over each scan block, in depth order.
__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const uint32_t* __restrict__ order, const uint32_t* __restrict__ touched,
              uint32_t count, uint32_t* __restrict__ block_sums) {
    __shared__ uint32_t wt[33];
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

// Exclusive scan of the block sums (one block), total instance count.
__global__ void __launch_bounds__(kSortThreads)
k_scan_blocks(uint32_t* __restrict__ block_sums, int nb, uint32_t cap, DevCounters* ctr) {
    __shared__ uint32_t wt[33];
    unsigned long long carry = 0;
    for (int base = 0; base < nb; base += kSortThreads * 4) {
        uint32_t v[4], s = 0;
        for (int k = 0; k < 4; ++k) {
            int i = base + threadIdx.x * 4 + k;
            v[k] = i < nb ? block_sums[i] : 0u;
            s += v[k];
        }
        uint32_t tot;
        uint32_t ex = block_exclusive_scan(s, wt, tot);
        unsigned long long run = carry + ex;
        for (int k = 0; k < 4; ++k) {
            int i = base + threadIdx.x * 4 + k;
            if (i < nb) block_sums[i] = (uint32_t)min(run, (unsigned long long)0xFFFFFFFFu);
            run += v[k];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        ctr->n_raw = carry;
        ctr->n_instances = (uint32_t)min(carry, (unsigned long long)cap);
        if (carry > cap) atomicOr(&ctr->status, (uint32_t)GS_DEV_CAPACITY);
    }
}

// Emit one instance per (Gaussian, tile in its rect), walking the depth
// order; tiles of a rect in row-major order.
__global__ void __launch_bounds__(kScanThreads)
k_emit(const uint32_t* __restrict__ order, const uint32_t* __restrict__ touched,
       const uint2* __restrict__ rects, const uint32_t* __restrict__ block_off, uint32_t count,
       int n, ViewTable vt, uint32_t cap, uint32_t* __restrict__ ikeys,
       uint32_t* __restrict__ ivals) {
    __shared__ uint32_t wt[33];
    const uint32_t start = blockIdx.x * (uint32_t)kScanTile;
    uint32_t vg[kScanItems], t[kScanItems], s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t i = start + threadIdx.x * kScanItems + k;
        vg[k] = i < count ? order[i] : 0u;
        t[k] = i < count ? touched[vg[k]] : 0u;
        s += t[k];
    }
    uint32_t tot;
    uint32_t off = block_exclusive_scan(s, wt, tot) + block_off[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        if (t[k] == 0u) continue;
        const int v = (int)(vg[k] / (uint32_t)n);
        const ViewGeom& geo = vt.v[v];
        const uint2 rc = rects[vg[k]];
        const int x0 = rc.x & 0xFFFF, y0 = rc.x >> 16, x1 = rc.y & 0xFFFF, y1 = rc.y >> 16;
        uint32_t pos = off;
        for (int ty = y0; ty < y1; ++ty) {
            const uint32_t row = (uint32_t)geo.tile_offset + (uint32_t)ty * geo.tiles_x;
            for (int tx = x0; tx < x1; ++tx, ++pos) {
                if (pos < cap) {
                    ikeys[pos] = row + (uint32_t)tx;
                    ivals[pos] = vg[k];
                }
            }
        }
        off += t[k];
    }
}

__global__ void k_ranges(const uint32_t* __restrict__ keys, const uint32_t* count_dev,
                         uint32_t* __restrict__ ranges) {
    const uint32_t count = *count_dev;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) ranges[2 * k] = i;
        if (i + 1 == count || keys[i + 1] != k) ranges[2 * k + 1] = i + 1;
    }
}

gs_status radix_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout,
                     const uint32_t* count_dev, uint32_t count_host, uint32_t cap, int shift,
                     int nb, uint32_t* hist, uint32_t* totals, cudaStream_t st) {
    k_radix_hist<<<nb, kSortThreads, 0, st>>>(kin, count_dev, count_host, cap, shift, nb, hist);
    k_radix_scan<<<kRadix, kSortThreads, 0, st>>>(hist, count_dev, count_host, cap, nb, totals);
    k_radix_scatter<<<nb, kSortThreads, 0, st>>>(kin, vin, kout, vout, count_dev, count_host,
                                                 cap, shift, nb, hist, totals);
    return launch_status();
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

    // 1. depth digits over the (view, Gaussian) pairs: 4 passes, A->B->A->B->A
    uint32_t* ka = buf<uint32_t>(p, ws, B_DKEY_A);
    uint32_t* va = buf<uint32_t>(p, ws, GS_BUF_DEPTH_ORDER);
    uint32_t* kb = buf<uint32_t>(p, ws, B_DKEY_B);
    uint32_t* vb = buf<uint32_t>(p, ws, B_DVAL_B);
    const int dnb = (int)((VN + kSortTile - 1) / kSortTile);
    for (int pass = 0; pass < 4; ++pass) {
        const bool even = (pass & 1) == 0;
        gs_status s = radix_pass(even ? ka : kb, even ? va : vb, even ? kb : ka, even ? vb : va,
                                 nullptr, VN, VN, pass * kRadixBits, dnb, hist, totals, st);
        if (s != GS_OK) return s;
    }

    // 2. scan of tiles touched in depth order, then emission
    const int snb = (int)((VN + kScanTile - 1) / kScanTile);
    uint32_t* bsums = buf<uint32_t>(p, ws, B_SCAN_BLOCKS);
    const uint32_t* touched = buf<uint32_t>(p, ws, GS_BUF_TOUCHED);
    k_scan_reduce<<<snb, kScanThreads, 0, st>>>(va, touched, VN, bsums);
    k_scan_blocks<<<1, kSortThreads, 0, st>>>(bsums, snb, icap, ctr);
    uint32_t* ika = buf<uint32_t>(p, ws, GS_BUF_TILE_KEYS);
    uint32_t* iva = buf<uint32_t>(p, ws, GS_BUF_TILE_VALUES);
    uint32_t* ikb = buf<uint32_t>(p, ws, B_IKEY_B);
    uint32_t* ivb = buf<uint32_t>(p, ws, B_IVAL_B);
    k_emit<<<snb, kScanThreads, 0, st>>>(va, touched, buf<uint2>(p, ws, GS_BUF_RECT), bsums, VN,
                                         n, p->vt, icap, ika, iva);
    gs_status s = launch_status();
    if (s != GS_OK) return s;

    // 3. tile-id digits over the instances
    const uint32_t* cnt = &ctr->n_instances;
    for (int pass = 0; pass < p->tile_passes; ++pass) {
        const bool even = (pass & 1) == 0;
        s = radix_pass(even ? ika : ikb, even ? iva : ivb, even ? ikb : ika, even ? ivb : iva, cnt,
                       0u, icap, pass * kRadixBits, p->inst_sort_blocks, hist, totals, st);
        if (s != GS_OK) return s;
    }
    const uint32_t* sorted_keys = (p->tile_passes & 1) ? ikb : ika;

    // 4. per-tile ranges
    uint32_t* ranges = buf<uint32_t>(p, ws, GS_BUF_RANGES);
    if (cudaMemsetAsync(ranges, 0, (size_t)p->total_tiles * 2 * sizeof(uint32_t), st) !=
        cudaSuccess)
        return GS_ERR_CUDA;
    k_ranges<<<kGrid, 256, 0, st>>>(sorted_keys, cnt, ranges);
    return launch_status();
}

}  // namespace gs
