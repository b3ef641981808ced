// Tile binning and per-tile depth sort (Sec. 3: "sorted based on the current
// camera depth"; the standard tile-splatting pipeline the paper builds on).
//
//  1. scan     exclusive prefix sum of tiles-touched per Gaussian (3 kernels,
//              fixed grid); total pair count M kept on the device, clamped to
//              the context capacity (overflow sets a status bit).
//  2. emit     pair j of Gaussian k: key = (tile << 32) | depth bits, value = k,
//              written in Gaussian order, so equal keys keep index order.
//  3. sort     stable LSD radix sort over the significant key bits, 8-bit
//              digits; each pass = block histograms, one scan over
//              (digit, block), stable scatter.  The grid is fixed (NB blocks,
//              each owning a contiguous chunk of ceil(M / NB) pairs) so that
//              no host synchronisation is needed to size it.
//  4. ranges   [start, end) of every tile in the sorted list.
// Result: total order (tile, depth key, Gaussian index), bit-exact.
#include "common.cuh"

#define SCAN_BLOCKS 1024
#define SORT_THREADS 256
#define SORT_ROWS 4
#define SORT_TILE (SORT_THREADS * SORT_ROWS)

// ---------------------------------------------------------------- scan
__global__ void k_scan_reduce(const uint32_t *__restrict__ x, int n, unsigned long long *bsum) {
    __shared__ unsigned long long s[256];
    const int chunk = (n + SCAN_BLOCKS - 1) / SCAN_BLOCKS;
    const int beg = blockIdx.x * chunk, end = min(beg + chunk, n);
    unsigned long long acc = 0;
    for (int i = beg + threadIdx.x; i < end; i += blockDim.x) acc += x[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = s[0];
}

__global__ void k_scan_blocks(unsigned long long *bsum, uint32_t *count, uint32_t cap, uint32_t *status) {
    __shared__ unsigned long long s[SCAN_BLOCKS];
    const int t = threadIdx.x;
    s[t] = bsum[t];
    __syncthreads();
    for (int off = 1; off < SCAN_BLOCKS; off <<= 1) {
        unsigned long long v = (t >= off) ? s[t - off] : 0ull;
        __syncthreads();
        s[t] += v;
        __syncthreads();
    }
    const unsigned long long incl = s[t];
    bsum[t] = incl - bsum[t];  // exclusive
    if (t == SCAN_BLOCKS - 1) {
        const unsigned long long total = incl;
        count[1] = (uint32_t)min(total, (unsigned long long)0xFFFFFFFFull);
        count[0] = (uint32_t)min(total, (unsigned long long)cap);
        if (total > cap) atomicOr(status, GS2_ST_CAPACITY);
    }
}

__global__ void k_scan_down(const uint32_t *__restrict__ x, int n, const unsigned long long *bsum, uint32_t cap,
                            uint32_t *offs) {
    __shared__ unsigned long long s[256];
    const int chunk = (n + SCAN_BLOCKS - 1) / SCAN_BLOCKS;
    const int beg = blockIdx.x * chunk, end = min(beg + chunk, n);
    unsigned long long base = bsum[blockIdx.x];
    for (int b0 = beg; b0 < end; b0 += 256) {
        const int i = b0 + threadIdx.x;
        const unsigned long long v = (i < end) ? x[i] : 0ull;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 256; off <<= 1) {
            unsigned long long a = (threadIdx.x >= off) ? s[threadIdx.x - off] : 0ull;
            __syncthreads();
            s[threadIdx.x] += a;
            __syncthreads();
        }
        if (i < end) offs[i] = (uint32_t)min(base + s[threadIdx.x] - v, (unsigned long long)cap);
        base += s[255];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- emit
// One CTA per 256 consecutive Gaussians: their pairs occupy one contiguous
// output range, which the CTA writes with all threads striding (coalesced,
// balanced even when one Gaussian covers thousands of tiles); a pair finds
// its Gaussian by binary search over the CTA's offsets in shared memory.
__global__ void __launch_bounds__(256) k_emit(ProjView pv, int n, int tiles_x, uint32_t cap,
                                              unsigned long long *keys, uint32_t *vals, unsigned long long *stats) {
    __shared__ uint32_t s_off[257];
    __shared__ uint2 s_rect[256];
    __shared__ uint32_t s_key[256];
    const int t = threadIdx.x;
    const int k = blockIdx.x * 256 + t;
    const uint32_t cnt = (k < n) ? pv.touched[k] : 0u;
    if (stats) {  // visible-Gaussian count, one atomic per warp
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, cnt != 0u);
        if ((t & 31) == 0 && b) atomicAdd(&stats[1], (unsigned long long)__popc(b));
    }
    const uint32_t off = (k < n) ? pv.offs[k] : 0u;
    s_off[t] = (k < n) ? off : 0xFFFFFFFFu;
    s_rect[t] = (k < n) ? pv.rect[k] : make_uint2(0u, 0u);
    s_key[t] = (k < n) ? pv.key[k] : 0u;
    const int last = min(n - 1, blockIdx.x * 256 + 255) - blockIdx.x * 256;
    __shared__ uint32_t s_beg, s_end;
    if (t == last) {
        s_end = min(off + cnt, cap);  // offsets are already clamped to cap
    }
    if (t == 0) s_beg = off;
    if (t == 0) s_off[256] = 0xFFFFFFFFu;
    __syncthreads();
    const uint32_t beg = s_beg, end = s_end;
    for (uint32_t j = beg + t; j < end; j += 256) {
        // largest i with s_off[i] <= j
        int lo = 0, hi = last;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= j) lo = mid;
            else hi = mid - 1;
        }
        const uint2 r = s_rect[lo];
        const uint32_t tx0 = r.x & 0xFFFFu, ty0 = r.x >> 16, tx1 = r.y & 0xFFFFu;
        const uint32_t wdt = tx1 - tx0, rel = j - s_off[lo];
        const uint32_t ty = ty0 + rel / wdt, tx = tx0 + rel % wdt;
        keys[j] = ((unsigned long long)(ty * (uint32_t)tiles_x + tx) << 32) | (unsigned long long)s_key[lo];
        vals[j] = (uint32_t)(blockIdx.x * 256 + lo);
    }
}

// ---------------------------------------------------------------- radix sort
__device__ __forceinline__ void chunk_of(uint32_t M, int nb, int b, uint32_t &beg, uint32_t &end) {
    const unsigned long long chunk = ((unsigned long long)M + nb - 1) / nb;
    const unsigned long long bb = min((unsigned long long)b * chunk, (unsigned long long)M);
    beg = (uint32_t)bb;
    end = (uint32_t)min(bb + chunk, (unsigned long long)M);
}

__global__ void __launch_bounds__(SORT_THREADS) k_hist(const unsigned long long *__restrict__ keys,
                                                       const uint32_t *count, int shift, uint32_t *ghist, int nb) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    uint32_t beg, end;
    chunk_of(count[0], nb, blockIdx.x, beg, end);
    for (uint32_t i = beg + threadIdx.x; i < end; i += SORT_THREADS)
        atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    ghist[threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Per-digit scan of the block histograms: CTA d turns row d of ghist (one count
// per sort block, coalesced) into exclusive prefixes and writes the digit's
// total; each scatter block adds the exclusive scan of the 256 digit totals.
__device__ __forceinline__ uint32_t block_excl_scan_1024(uint32_t v, uint32_t *swarp, uint32_t &total) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) swarp[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t z = lane < nw ? swarp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < nw) swarp[lane] = z;
    }
    __syncthreads();
    total = swarp[(blockDim.x >> 5) - 1];
    const uint32_t before = (w > 0) ? swarp[w - 1] : 0u;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(1024) k_digit_scan(uint32_t *ghist, int nb, uint32_t *dtot) {
    __shared__ uint32_t swarp[32];
    const int d = blockIdx.x, t = threadIdx.x;
    const uint32_t v = (t < nb) ? ghist[d * nb + t] : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan_1024(v, swarp, tot);
    if (t < nb) ghist[d * nb + t] = ex;
    if (t == 0) dtot[d] = tot;
}

__global__ void __launch_bounds__(SORT_THREADS) k_scatter(const unsigned long long *__restrict__ kin,
                                                          const uint32_t *__restrict__ vin,
                                                          unsigned long long *__restrict__ kout,
                                                          uint32_t *__restrict__ vout, const uint32_t *count,
                                                          int shift, const uint32_t *ghist, int nb,
                                                          const uint32_t *dtot) {
    __shared__ uint32_t s_off[256];
    __shared__ uint32_t s_wc[SORT_THREADS / 32][256];
    __shared__ uint32_t swarp[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t beg, end;
    chunk_of(count[0], nb, blockIdx.x, beg, end);
    {
        uint32_t tot;
        const uint32_t base = block_excl_scan_1024(dtot[t], swarp, tot);
        s_off[t] = base + ghist[t * nb + blockIdx.x];
    }
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (uint32_t base = beg; base < end; base += SORT_TILE) {
#pragma unroll
        for (int i = 0; i < SORT_THREADS / 32; ++i) s_wc[i][t] = 0u;
        __syncthreads();
        unsigned long long key[SORT_ROWS];
        uint32_t val[SORT_ROWS], dig[SORT_ROWS], pos[SORT_ROWS];
#pragma unroll
        for (int r = 0; r < SORT_ROWS; ++r) {
            const uint32_t idx = base + (uint32_t)(w * (32 * SORT_ROWS) + r * 32 + lane);
            const bool valid = idx < end;
            key[r] = valid ? kin[idx] : 0ull;
            val[r] = valid ? vin[idx] : 0u;
            dig[r] = valid ? ((uint32_t)(key[r] >> shift) & 255u) : 256u;
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, dig[r]);
            const uint32_t rank = __popc(peers & lt_mask);
            uint32_t cnt = 0u;
            if (valid) cnt = s_wc[w][dig[r]];
            __syncwarp();
            if (valid && rank == 0u) s_wc[w][dig[r]] = cnt + __popc(peers);
            __syncwarp();
            pos[r] = cnt + rank;
        }
        __syncthreads();
        uint32_t run = 0u;
#pragma unroll
        for (int i = 0; i < SORT_THREADS / 32; ++i) {
            const uint32_t c = s_wc[i][t];
            s_wc[i][t] = run;
            run += c;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < SORT_ROWS; ++r) {
            if (dig[r] < 256u) {
                const uint32_t dst = s_off[dig[r]] + s_wc[w][dig[r]] + pos[r];
                kout[dst] = key[r];
                vout[dst] = val[r];
            }
        }
        __syncthreads();
        s_off[t] += run;
        __syncthreads();
    }
}

__global__ void k_ranges(const unsigned long long *__restrict__ keys, const uint32_t *count, uint2 *ranges,
                         unsigned long long *stats) {
    const uint32_t M = count[0];
    if (stats && blockIdx.x == 0 && threadIdx.x == 0) {
        stats[0] += M;
        stats[2] += 1ull;
    }
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < M; j += gridDim.x * blockDim.x) {
        const uint32_t tile = (uint32_t)(keys[j] >> 32);
        if (j == 0u || (uint32_t)(keys[j - 1] >> 32) != tile) ranges[tile].x = j;
        if (j == M - 1u || (uint32_t)(keys[j + 1] >> 32) != tile) ranges[tile].y = j + 1u;
    }
}

cudaError_t launch_bin_sort(gs2_ctx *ctx, ProjView pv, int n, int tiles_x, int tiles_y, cudaStream_t st,
                            unsigned long long *stats) {
    const uint32_t cap = (uint32_t)ctx->max_pairs;
    unsigned long long *bsum = (unsigned long long *)ctx->bsum;
    k_scan_reduce<<<SCAN_BLOCKS, 256, 0, st>>>(pv.touched, n, bsum);
    k_scan_blocks<<<1, SCAN_BLOCKS, 0, st>>>(bsum, ctx->d_count, cap, ctx->d_status);
    k_scan_down<<<SCAN_BLOCKS, 256, 0, st>>>(pv.touched, n, bsum, cap, pv.offs);
    if (n > 0) k_emit<<<(n + 255) / 256, 256, 0, st>>>(pv, n, tiles_x, cap, ctx->keys[0], ctx->vals[0], stats);
    const int ntiles = tiles_x * tiles_y;
    int tile_bits = 0;
    while ((1 << tile_bits) < ntiles) ++tile_bits;
    const int bits = 32 + tile_bits;
    const int passes = (bits + 7) / 8;
    const int nb = ctx->nb_sort;
    uint32_t *dtot = ctx->ghist + 256 * nb;   // 256 digit totals after the histogram table
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_hist<<<nb, SORT_THREADS, 0, st>>>(ctx->keys[cur], ctx->d_count, shift, ctx->ghist, nb);
        k_digit_scan<<<256, 1024, 0, st>>>(ctx->ghist, nb, dtot);
        k_scatter<<<nb, SORT_THREADS, 0, st>>>(ctx->keys[cur], ctx->vals[cur], ctx->keys[cur ^ 1],
                                               ctx->vals[cur ^ 1], ctx->d_count, shift, ctx->ghist, nb, dtot);
        cur ^= 1;
    }
    ctx->sorted = cur;
    cudaError_t e = cudaMemsetAsync(ctx->ranges, 0, sizeof(uint2) * (size_t)ntiles, st);
    if (e != cudaSuccess) return e;
    k_ranges<<<148 * 4, 256, 0, st>>>(ctx->keys[cur], ctx->d_count, ctx->ranges, stats);
    GS2_COUNT_LAUNCH(3 + (n > 0) + 3 * passes + 1);
    return cudaGetLastError();
}
