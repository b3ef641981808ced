// Tile binning and per-tile depth sort (Sec. 3: "sorted based on the current
// camera depth"; the standard tile-splatting pipeline the paper builds on).
//
//  1. depth   stable LSD radix sort of the Gaussians by FP32 depth bits (4
//             passes over n; Gaussians that touch no tile get the largest key
//             and sort last) -> rank order (key, index);
//  2. scan    exclusive prefix sum of tiles-touched in rank order, one kernel
//             (decoupled look-back over chunks of ranks); total pair count M
//             on the device, clamped to the context capacity (overflow sets a
//             status bit);
//  3. emit    pairs (tile id, Gaussian id) in rank order, one CTA per 256
//             ranks; a tile of a Gaussian's rectangle that its support
//             ellipse misses gets the key ntiles (a dropped pair);
//  4. tiles   stable LSD radix sort of the live pairs by tile id
//             (ceil(tile bits / 8) passes of equal width, 2 of 7 and 6 bits at
//             1600x1040); the first pass drops the dead pairs (neither counted
//             nor written), so the second sorts the listed pairs only --
//             stability keeps rank order per tile;
//  5. ranges  [start, end) of every tile in the sorted list.
// Result: total order (tile, depth key, Gaussian index), bit-exact.  Each
// radix pass = block histograms over a fixed grid of NB CTAs (each owning a
// contiguous chunk), a per-digit scan, and a stable scatter; element counts
// live on the device, so no host synchronisation sizes anything.  The scan's
// wait on an earlier chunk's look-back word is bounded: past the limit it sets
// GS2_ST_TIMEOUT and goes on (the result is then wrong but every access stays
// in bounds); with chunks claimed in order the wait cannot block, since a
// claimed chunk publishes its sum before it waits.
// (Measured and not kept: the same one-kernel look-back pass for every radix
// pass, fed with digit counts gathered by the emission -- 2x slower per pass,
// each 1024-key tile exposing its load and a look-back chain.)
#include "common.cuh"

#define SORT_THREADS 256

// ---------------------------------------------------------------- look-back words
// 64-bit words written and read whole (single-copy atomic): a flag (the
// aggregate of one unit, or the inclusive prefix up to it) and a value.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
#define LB_SPIN_LIMIT (1u << 20)   // polls of one look-back window before giving up (about a second)

// Look-back of chunk c > 0 over the states of the earlier chunks, by one full
// warp: lane i reads chunk j0 - i (a chunk before 0 reads as an inclusive
// prefix of 0); the sums of the chunks after the nearest inclusive prefix and
// that prefix give c's exclusive prefix.  A window with an unpublished chunk
// is read again, at most `limit` times in a row (with a short sleep after the
// first 32); past that the wait gives up and the function returns false with a
// partial sum.  Returns the exclusive prefix in excl (every lane).
__device__ __forceinline__ bool scan_lookback(const unsigned long long *state, int c, uint32_t limit,
                                              unsigned long long &excl) {
    const int lane = threadIdx.x & 31;
    excl = 0;
    int j0 = c - 1;
    uint32_t spins = 0;
    for (;;) {
        const int j = j0 - lane;
        const unsigned long long v = j >= 0 ? ld_relaxed_u64(&state[j]) : (2ull << 62);
        const uint32_t flag = (uint32_t)(v >> 62);
        const uint32_t pre = __ballot_sync(0xFFFFFFFFu, flag == 2u);
        const int lim = pre ? __ffs(pre) - 1 : 31;   // lanes 0..lim are needed
        const uint32_t need = lim == 31 ? 0xFFFFFFFFu : ((2u << lim) - 1u);
        if (__ballot_sync(0xFFFFFFFFu, flag == 0u) & need) {   // some not published yet
            if (++spins > limit) return false;
            if (spins > 32) __nanosleep(64);
            continue;
        }
        unsigned long long part = lane <= lim ? (v & ((1ull << 62) - 1)) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
        excl += part;
        if (pre) return true;
        j0 -= 32;
        spins = 0;
    }
}

// ---------------------------------------------------------------- scan
// Exclusive prefix sum of tiles-touched in rank order, in one pass: chunk c
// (claimed in order by ticket) of `chunk` consecutive ranks gathers touched
// in rank order into tsort, publishes its sum, adds the sums of the earlier
// chunks (look-back until an inclusive prefix, one warp reading 32 chunks at
// a time), publishes its own inclusive prefix, and writes its offsets
// (clamped to cap).  The last chunk writes the pair count.  States: GS2_SCAN_CHUNKS 64-bit words (bits 63..62: 1 sum, 2
// inclusive prefix), zero at the start, as is the chunk ticket.
#define TS_THREADS 256
#define TS_ITEMS 16
#define TS_ROUND (TS_THREADS * TS_ITEMS)
#define TS_PAD(j) ((j) + ((j) >> 5))
__device__ __forceinline__ unsigned long long block_excl_scan64(unsigned long long v, unsigned long long *swarp,
                                                                unsigned long long &total) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) swarp[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long z = lane < (TS_THREADS >> 5) ? swarp[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < (TS_THREADS >> 5)) swarp[lane] = z;
    }
    __syncthreads();
    total = swarp[(TS_THREADS >> 5) - 1];
    const unsigned long long before = (w > 0) ? swarp[w - 1] : 0ull;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(TS_THREADS) k_touch_scan(ProjView pv, const uint32_t *__restrict__ order, int n,
                                                           int chunk, uint32_t cap, uint32_t *count,
                                                           uint32_t *status, uint32_t *ss) {
    __shared__ uint32_t s_v[TS_PAD(TS_ROUND)];
    __shared__ unsigned long long swarp[TS_THREADS / 32];
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_c;
    const int t = threadIdx.x;
    unsigned long long *state = reinterpret_cast<unsigned long long *>(ss + GS2_SS_CHUNKS);
    if (t == 0) s_c = atomicAdd(&ss[GS2_SS_TICKET], 1u);
    __syncthreads();
    const int c = (int)s_c;
    const int beg = c * chunk, end = min(n, beg + chunk);
    // the chunk's sum, gathering tsort on the way (coalesced writes)
    unsigned long long acc = 0;
    for (int r = beg + t; r < end; r += TS_THREADS) {
        const uint32_t v = pv.touched[order[r]];
        pv.tsort[r] = v;
        acc += v;
    }
    unsigned long long agg;
    block_excl_scan64(acc, swarp, agg);
    // warp 0 publishes the chunk's sum and looks back over the earlier chunks
    if (t < 32) {
        unsigned long long excl = 0;
        if (c == 0) {
            if (t == 0) st_relaxed_u64(&state[0], (2ull << 62) | agg);
        } else {
            if (t == 0) st_relaxed_u64(&state[c], (1ull << 62) | agg);
            if (!scan_lookback(state, c, LB_SPIN_LIMIT, excl) && t == 0) atomicOr(status, GS2_ST_TIMEOUT);
            if (t == 0) st_relaxed_u64(&state[c], (2ull << 62) | (excl + agg));
        }
        if (t == 0) s_base = excl;
    }
    __syncthreads();
    // offsets: rounds of TS_ROUND ranks, read back coalesced, transposed so
    // that each thread scans TS_ITEMS consecutive ranks
    unsigned long long base = s_base;
    for (int r0 = beg; r0 < end; r0 += TS_ROUND) {
#pragma unroll
        for (int i = 0; i < TS_ITEMS; ++i) {
            const int j = i * TS_THREADS + t;
            s_v[TS_PAD(j)] = (r0 + j < end) ? pv.tsort[r0 + j] : 0u;
        }
        __syncthreads();
        uint32_t x[TS_ITEMS];
        unsigned long long sum = 0;
#pragma unroll
        for (int i = 0; i < TS_ITEMS; ++i) {
            x[i] = s_v[TS_PAD(t * TS_ITEMS + i)];
            sum += x[i];
        }
        unsigned long long tot;
        unsigned long long run = base + block_excl_scan64(sum, swarp, tot);
#pragma unroll
        for (int i = 0; i < TS_ITEMS; ++i) {
            s_v[TS_PAD(t * TS_ITEMS + i)] = (uint32_t)min(run, (unsigned long long)cap);
            run += x[i];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < TS_ITEMS; ++i) {
            const int j = i * TS_THREADS + t;
            if (r0 + j < end) pv.offs[r0 + j] = s_v[TS_PAD(j)];
        }
        __syncthreads();
        base += tot;
    }
    if (end == n && t == 0) {   // the last chunk: the pair count
        const unsigned long long total = base;
        count[1] = (uint32_t)min(total, (unsigned long long)0xFFFFFFFFull);
        count[0] = (uint32_t)min(total, (unsigned long long)cap);
        if (total > cap) atomicOr(status, GS2_ST_CAPACITY);
    }
}

// ---------------------------------------------------------------- depth keys
// key = FP32 depth bits of every Gaussian (positive FP32 bit patterns order
// like the values; depths behind the near plane sort after them and touch no
// tile), value = index.  Sorting all Gaussians, not only those on screen,
// makes the order depend on the means and the camera alone, so a sweep can
// reuse it for every group that does not move the means.  Thread 0 also
// publishes the element count n for the radix passes.
__global__ void k_depth_keys(ProjView pv, int n, uint32_t *count_slot) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0) *count_slot = (uint32_t)n;
    if (k >= n) return;
    pv.dk[0][k] = pv.key[k];
    pv.dv[0][k] = (uint32_t)k;
}

// ---------------------------------------------------------------- emit
// One CTA per 256 consecutive ranks: their pairs (one per tile of each
// Gaussian's rectangle) occupy one contiguous output range, which the CTA
// writes with all threads striding (coalesced, balanced even when one Gaussian
// covers thousands of tiles); a pair finds its rank by binary search over the
// CTA's offsets in shared memory.  A tile of the rectangle that the Gaussian's
// support ellipse does not reach gets the key ntiles: it sorts after every
// tile and the range pass leaves it out of the lists, so the compositing and
// the accumulation never walk it.  The tile test is the reproducible FP32
// support_reaches of decide.cuh, so the lists are a function of the FP32
// parameters and camera alone, bit for bit.
// ids_emit (deterministic mode, else NULL): the pair's value is its emission
// index j and its Gaussian id goes to ids_emit[j] (0xFFFFFFFF for a dropped
// pair), so that after the tile sort every pair's sorted position can be
// mapped back to its emission slot.
__global__ void __launch_bounds__(256) k_emit(ProjView pv, const uint32_t *__restrict__ order, int n, int tiles_x,
                                              uint32_t ntiles, uint32_t cap, uint32_t *keys, uint32_t *vals,
                                              unsigned long long *stats, uint32_t *__restrict__ ids_emit) {
    __shared__ uint32_t s_off[256];
    __shared__ uint2 s_rect[256];
    __shared__ SupportRows s_sr[256];
    __shared__ uint32_t s_id[256];
    __shared__ uint32_t s_row[256];    // exclusive prefix of the rectangles' tile rows over the CTA's ranks
    __shared__ uint32_t s_wsum[8];
    __shared__ uint32_t s_end, s_rows;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int r = blockIdx.x * 256 + t;
    const uint32_t id = (r < n) ? order[r] : 0u;
    const uint32_t cnt = (r < n) ? pv.tsort[r] : 0u;
    if (stats) {  // visible-Gaussian count, one atomic per warp
        const uint32_t b = __ballot_sync(0xFFFFFFFFu, cnt != 0u);
        if (lane == 0 && b) atomicAdd(&stats[1], (unsigned long long)__popc(b));
    }
    const uint32_t off = (r < n) ? pv.offs[r] : 0u;
    s_off[t] = off;
    const uint2 rc = (cnt != 0u) ? pv.rect[id] : make_uint2(0u, 0u);   // only ranks with pairs are looked up
    s_rect[t] = rc;
    s_id[t] = id;
    if (cnt != 0u) {
        const float4 A = pv.recA[id];
        s_sr[t] = support_rows(A.x, A.y, A.z, A.w, pv.k2[id], pv.col[id].w);
    }
    // tile rows of this rank's rectangle (its pairs are row-major in it)
    const uint32_t h = cnt != 0u ? (rc.y >> 16) - (rc.x >> 16) : 0u;
    uint32_t inc = h;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += v;
    }
    if (lane == 31) s_wsum[w] = inc;
    const int last = min(n - 1, blockIdx.x * 256 + 255) - blockIdx.x * 256;
    if (t == last) s_end = min(off + cnt, cap);   // offsets are already clamped to cap
    __syncthreads();
    uint32_t wbase = 0u, tot = 0u;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint32_t v = s_wsum[q];
        wbase += q < w ? v : 0u;
        tot += v;
    }
    s_row[t] = wbase + inc - h;
    if (t == 0) s_rows = tot;
    __syncthreads();
    const uint32_t end = s_end, nrows = s_rows;
    // one (rank, tile row) per thread and step: the support's column range in
    // that band once, then the row's tiles in order
    for (uint32_t u = t; u < nrows; u += 256) {
        int lo = 0, hi = last;   // largest i with s_row[i] <= u (a rank with rows)
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_row[mid] <= u) lo = mid;
            else hi = mid - 1;
        }
        const uint2 rr = s_rect[lo];
        const uint32_t tx0 = rr.x & 0xFFFFu, ty0 = rr.x >> 16, tx1 = rr.y & 0xFFFFu;
        const uint32_t wdt = tx1 - tx0, row = u - s_row[lo];
        const uint32_t base = s_off[lo] + row * wdt;
        if (base >= end) continue;
        const uint32_t ty = ty0 + row, gid = s_id[lo];
        const SupportRow band = support_row(s_sr[lo], (float)(ty * GS2_TILE), (float)GS2_TILE);
        const uint32_t m = min(wdt, end - base);
        for (uint32_t c = 0; c < m; ++c) {
            const uint32_t j = base + c, tx = tx0 + c;
            const bool live = support_row_reaches(band, (float)(tx * GS2_TILE), (float)GS2_TILE);
            keys[j] = live ? ty * (uint32_t)tiles_x + tx : ntiles;
            if (ids_emit) {
                vals[j] = j;
                ids_emit[j] = live ? gid : 0xFFFFFFFFu;
            } else {
                vals[j] = gid;
            }
        }
    }
}

// Deterministic mode, after the tile sort (values = emission indices):
// list[s] = Gaussian id of sorted pair s, inv[j] = sorted position of emitted
// pair j (dropped pairs have no sorted position: ids_emit[j] = 0xFFFFFFFF
// marks them).  count[3]: the listed pairs.
__global__ void k_det_gather(const uint32_t *__restrict__ sorted_vals, const uint32_t *__restrict__ ids_emit,
                             const uint32_t *count, uint32_t *__restrict__ list, uint32_t *__restrict__ inv) {
    const uint32_t M = count[3];
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < M; s += gridDim.x * blockDim.x) {
        const uint32_t j = sorted_vals[s];
        list[s] = ids_emit[j];
        inv[j] = s;
    }
}

// ---------------------------------------------------------------- radix sort (32-bit keys, 32-bit values)
__device__ __forceinline__ void chunk_of(uint32_t M, int nb, int b, uint32_t &beg, uint32_t &end) {
    const unsigned long long chunk = ((unsigned long long)M + nb - 1) / nb;
    const unsigned long long bb = min((unsigned long long)b * chunk, (unsigned long long)M);
    beg = (uint32_t)bb;
    end = (uint32_t)min(bb + chunk, (unsigned long long)M);
}

// keys >= dead_from (dropped pairs) are not counted
__global__ void __launch_bounds__(SORT_THREADS) k_hist(const uint32_t *__restrict__ keys, const uint32_t *count,
                                                       int shift, uint32_t mask, uint32_t *ghist, int nb,
                                                       uint32_t dead_from) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    uint32_t beg, end;
    chunk_of(*count, nb, blockIdx.x, beg, end);
    for (uint32_t i = beg + threadIdx.x; i < end; i += SORT_THREADS) {
        const uint32_t k = keys[i];
        if (k < dead_from) atomicAdd(&h[(k >> shift) & mask], 1u);
    }
    __syncthreads();
    ghist[threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Per-digit scan of the block histograms: CTA d turns row d of ghist (one count
// per sort block, coalesced) into exclusive prefixes and writes the digit's
// total; each scatter block adds the exclusive scan of the 256 digit totals.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *swarp, uint32_t &total) {
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
    const uint32_t ex = block_excl_scan(v, swarp, tot);
    if (t < nb) ghist[d * nb + t] = ex;
    if (t == 0) dtot[d] = tot;
}

// ROWS keys per thread per 256-thread round (a tuning parameter: 2, 4, 8 or 16).
// Keys >= dead_from (dropped pairs) are neither ranked nor written;
// count_live (or NULL) receives the number of the others, the element count
// of the following passes.
template <int ROWS>
__global__ void __launch_bounds__(SORT_THREADS) k_scatter(const uint32_t *__restrict__ kin,
                                                          const uint32_t *__restrict__ vin,
                                                          uint32_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                                          const uint32_t *count, int shift, uint32_t mask,
                                                          const uint32_t *ghist, int nb, const uint32_t *dtot,
                                                          uint32_t dead_from, uint32_t *count_live) {
    constexpr int SORT_TILE = SORT_THREADS * ROWS;
    __shared__ uint32_t s_off[256];
    __shared__ uint32_t s_wc[SORT_THREADS / 32][256];
    __shared__ uint32_t s_lb[256];                       // tile-local start of each digit
    __shared__ uint32_t s_k[SORT_TILE], s_v[SORT_TILE];  // the tile, stably sorted by digit
    __shared__ uint32_t swarp[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t beg, end;
    chunk_of(*count, nb, blockIdx.x, beg, end);
    {
        uint32_t tot;
        const uint32_t base = block_excl_scan(dtot[t], swarp, tot);
        s_off[t] = base + ghist[t * nb + blockIdx.x];
        if (count_live && blockIdx.x == 0 && t == 0) *count_live = tot;
    }
    const uint32_t lt_mask = (1u << lane) - 1u;
    // the next tile's keys and values are loaded while this one is ranked and written
    uint32_t nkey[ROWS], nval[ROWS];
    auto load_tile = [&](uint32_t b0) {
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const uint32_t idx = b0 + (uint32_t)(w * (32 * ROWS) + r * 32 + lane);
            nkey[r] = idx < end ? kin[idx] : 0u;
            nval[r] = idx < end ? vin[idx] : 0u;
        }
    };
    load_tile(beg);
    for (uint32_t base = beg; base < end; base += SORT_TILE) {
        uint32_t key[ROWS], val[ROWS], dig[ROWS], pos[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            key[r] = nkey[r];
            val[r] = nval[r];
        }
        if (base + SORT_TILE < end) load_tile(base + SORT_TILE);
#pragma unroll
        for (int i = 0; i < SORT_THREADS / 32; ++i) s_wc[i][t] = 0u;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            const uint32_t idx = base + (uint32_t)(w * (32 * ROWS) + r * 32 + lane);
            const bool valid = idx < end && key[r] < dead_from;
            dig[r] = valid ? ((key[r] >> shift) & mask) : 256u;
            // lanes with the same digit value (256 marks a slot past the end)
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
        uint32_t tile_n;
        s_lb[t] = block_excl_scan(run, swarp, tile_n);
        __syncthreads();
        // local stable sort of the tile by digit in shared memory ...
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
            if (dig[r] < 256u) {
                const uint32_t li = s_lb[dig[r]] + s_wc[w][dig[r]] + pos[r];
                s_k[li] = key[r];
                s_v[li] = val[r];
            }
        }
        __syncthreads();
        // ... then consecutive threads write consecutive positions of each digit's run
        for (uint32_t i = t; i < tile_n; i += SORT_THREADS) {
            const uint32_t kk = s_k[i], d = (kk >> shift) & mask;
            const uint32_t dst = s_off[d] + (i - s_lb[d]);
            kout[dst] = kk;
            vout[dst] = s_v[i];
        }
        __syncthreads();
        s_off[t] += run;
        __syncthreads();
    }
}

// `bits` significant key bits, ping-pong between (k[0], v[0]) and (k[1], v[1]);
// returns the index of the buffer holding the result.  The passes split the
// bits evenly (13 tile bits: 7 + 6, not 8 + 5): a digit of fewer values
// leaves longer runs of equal digits in each radix tile, so the scatter's
// stores cover fewer memory segments.  Keys >= dead_from are dropped by the
// first pass, which writes the number of the others to count_live (the count
// of the later passes); count_live = NULL: count for every pass.
static int radix_sort(uint32_t *k[2], uint32_t *v[2], const uint32_t *count, int bits, uint32_t *ghist, int nb,
                      int rows, cudaStream_t st, int *launches, uint32_t dead_from = 0xFFFFFFFFu,
                      uint32_t *count_live = nullptr) {
    uint32_t *dtot = ghist + 256 * nb;
    int cur = 0;
    const int passes = (bits + 7) / 8;
    const int width = (bits + passes - 1) / passes;
    const uint32_t mask = (1u << width) - 1u;
    for (int p = 0; p < passes; ++p) {
        const int shift = width * p;
        const uint32_t *cnt = (p > 0 && count_live) ? count_live : count;
        const uint32_t dead = p == 0 ? dead_from : 0xFFFFFFFFu;
        uint32_t *live = p == 0 ? count_live : nullptr;
        k_hist<<<nb, SORT_THREADS, 0, st>>>(k[cur], cnt, shift, mask, ghist, nb, dead);
        k_digit_scan<<<256, 1024, 0, st>>>(ghist, nb, dtot);
#define GS2_SCATTER(R)                                                                                            \
    k_scatter<R><<<nb, SORT_THREADS, 0, st>>>(k[cur], v[cur], k[cur ^ 1], v[cur ^ 1], cnt, shift, mask, ghist, nb,  \
                                              dtot, dead, live)
        if (rows == 2) GS2_SCATTER(2);
        else if (rows == 8) GS2_SCATTER(8);
        else if (rows == 16) GS2_SCATTER(16);
        else GS2_SCATTER(4);
#undef GS2_SCATTER
        cur ^= 1;
    }
    *launches += 3 * passes;
    return cur;
}

// [start, end) of every tile: each thread checks four consecutive sorted keys
// (one 16-byte load when aligned) against their successors.  count[3]: the
// listed pairs (the tile sort dropped the pairs whose tile the support
// ellipse misses); count[0]: the emitted pairs (statistics).
__global__ void k_ranges(const uint32_t *__restrict__ keys, const uint32_t *count, uint2 *ranges, uint32_t ntiles,
                         unsigned long long *stats) {
    const uint32_t M = count[3];
    if (stats && blockIdx.x == 0 && threadIdx.x == 0) {   // atomic: concurrent views share the counters
        atomicAdd(&stats[0], (unsigned long long)count[0]);
        atomicAdd(&stats[2], 1ull);
    }
    // listed pairs: the end of the last tile (pairs past it are not tiles)
    const uint32_t nq = (M + 3u) / 4u;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const uint32_t j0 = 4u * q;
        uint32_t k[5];
        if (j0 + 4u <= M) {
            const uint4 v = reinterpret_cast<const uint4 *>(keys)[q];
            k[0] = v.x; k[1] = v.y; k[2] = v.z; k[3] = v.w;
        } else {
            for (int i = 0; i < 4; ++i) k[i] = (j0 + i < M) ? keys[j0 + i] : 0u;
        }
        k[4] = (j0 + 4u < M) ? keys[j0 + 4u] : 0u;
        if (j0 == 0u && k[0] < ntiles) ranges[k[0]].x = 0u;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint32_t j = j0 + i;
            if (j >= M) break;
            if (j + 1u == M) {
                if (k[i] < ntiles) ranges[k[i]].y = M;
            } else if (k[i + 1] != k[i]) {
                if (k[i] < ntiles) ranges[k[i]].y = j + 1u;
                if (k[i + 1] < ntiles) ranges[k[i + 1]].x = j + 1u;
            }
            if (stats && k[i] < ntiles && (j + 1u == M || k[i + 1] >= ntiles))
                atomicAdd(&stats[4], (unsigned long long)(j + 1u));
        }
    }
}

// Launch order of the tiles for the compositing and the accumulation: by
// descending list length, in buckets of floor(log2(length)) (order within a
// bucket arbitrary, empty tiles last), so the longest tiles start in the
// first waves and the last wave is short.  The order changes no result: tiles
// are independent.  One CTA: a shared-memory histogram of the buckets, a scan,
// and a scatter by shared atomics.
__global__ void __launch_bounds__(1024) k_tile_order(const uint2 *__restrict__ ranges, int ntiles,
                                                     uint32_t *__restrict__ order) {
    __shared__ uint32_t cnt[33];
    const int t = threadIdx.x;
    if (t < 33) cnt[t] = 0u;
    __syncthreads();
    auto bucket = [&](int i) {
        const uint2 r = ranges[i];
        const uint32_t len = r.y - r.x;
        return len ? (uint32_t)__clz(len) : 32u;   // 0 for the longest lists, 32 for empty tiles
    };
    for (int i = t; i < ntiles; i += blockDim.x) atomicAdd(&cnt[bucket(i)], 1u);
    __syncthreads();
    if (t == 0) {
        uint32_t acc = 0u;
        for (int b = 0; b < 33; ++b) {
            const uint32_t c = cnt[b];
            cnt[b] = acc;
            acc += c;
        }
    }
    __syncthreads();
    for (int i = t; i < ntiles; i += blockDim.x) order[atomicAdd(&cnt[bucket(i)], 1u)] = (uint32_t)i;
}

// Test of the bounded wait (no GPU fault): one warp looks back from chunk c
// over states that nothing publishes (zeroed by the caller), gives up after
// `limit` polls and sets GS2_ST_TIMEOUT, as the scan does when a wait runs out.
__global__ void k_debug_lookback(const unsigned long long *state, int c, uint32_t limit, uint32_t *status) {
    unsigned long long excl;
    const bool ok = scan_lookback(state, c, limit, excl);
    if (!ok && threadIdx.x == 0) atomicOr(status, GS2_ST_TIMEOUT);
}

cudaError_t launch_debug_lookback(gs2_ctx *ctx, int c, uint32_t limit, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ctx->sort_state, 0, sizeof(uint32_t) * GS2_SS_WORDS, st);
    if (e != cudaSuccess) return e;
    k_debug_lookback<<<1, 32, 0, st>>>(reinterpret_cast<const unsigned long long *>(ctx->sort_state + GS2_SS_CHUNKS),
                                       c, limit, ctx->d_status);
    GS2_COUNT_LAUNCH(1);
    return cudaGetLastError();
}

cudaError_t launch_bin_sort(gs2_ctx *ctx, ProjView pv, int n, int tiles_x, int tiles_y, cudaStream_t st,
                            unsigned long long *stats, const uint32_t *order_in, uint32_t *order_out) {
    const uint32_t cap = (uint32_t)ctx->max_pairs;
    const int nb = ctx->nb_sort;
    int launches = 0;
    const int ntiles = tiles_x * tiles_y;
    cudaError_t e = cudaMemsetAsync(ctx->ranges, 0, sizeof(uint2) * (size_t)ntiles, st);
    if (e != cudaSuccess) return e;
    const bool det = ctx->cfg.deterministic != 0 && ctx->det_part;
    if (n == 0) {
        ctx->sorted = 0;
        ctx->list_ids = ctx->vals[0];
        ctx->det_order = nullptr;
        if (ctx->tile_order) {   // every tile empty: any order
            k_tile_order<<<1, 1024, 0, st>>>(ctx->ranges, ntiles, ctx->tile_order);
            GS2_COUNT_LAUNCH(1);
        }
        return cudaMemsetAsync(ctx->d_count, 0, sizeof(uint32_t) * 4, st);
    }
    // the scan's chunk ticket and look-back states start at zero
    e = cudaMemsetAsync(ctx->sort_state, 0, sizeof(uint32_t) * GS2_SS_WORDS, st);
    if (e != cudaSuccess) return e;
    // 1. depth order of the Gaussians (or the caller's copy of it for the same
    //    means and camera)
    const uint32_t *order = order_in;
    if (!order) {
        k_depth_keys<<<(n + 255) / 256, 256, 0, st>>>(pv, n, ctx->d_count + 2);
        ++launches;
        const int dcur =
            radix_sort(pv.dk, pv.dv, ctx->d_count + 2, 32, ctx->ghist, nb, ctx->sort_rows, st, &launches);
        order = pv.dv[dcur];
        if (order_out) {
            e = cudaMemcpyAsync(order_out, order, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return e;
        }
    }
    // 2. tiles-touched in rank order, exclusive scan -> pair offsets and the pair count
    const int chunk = ((n + GS2_SCAN_CHUNKS - 1) / GS2_SCAN_CHUNKS + TS_ROUND - 1) / TS_ROUND * TS_ROUND;
    k_touch_scan<<<(n + chunk - 1) / chunk, TS_THREADS, 0, st>>>(pv, order, n, chunk, cap, ctx->d_count,
                                                                 ctx->d_status, ctx->sort_state);
    // 3. pairs in rank order
    k_emit<<<(n + 255) / 256, 256, 0, st>>>(pv, order, n, tiles_x, (uint32_t)ntiles, cap, ctx->keys[0],
                                            ctx->vals[0], stats, det ? ctx->det_ids : nullptr);
    // 4. stable sort of the live pairs by tile id (keys 0..ntiles - 1; ntiles: dropped by the first pass)
    ctx->sorted = radix_sort(ctx->keys, ctx->vals, ctx->d_count, gs2_tile_bits(ntiles), ctx->ghist, nb,
                             ctx->sort_rows, st, &launches, (uint32_t)ntiles, ctx->d_count + 3);
    ctx->list_ids = ctx->vals[ctx->sorted];
    ctx->det_order = order;
    if (det) {
        k_det_gather<<<148 * 4, 256, 0, st>>>(ctx->vals[ctx->sorted], ctx->det_ids, ctx->d_count, ctx->det_list,
                                              ctx->det_inv);
        ctx->list_ids = ctx->det_list;
        ++launches;
    }
    // 5. tile ranges
    k_ranges<<<148 * 4, 256, 0, st>>>(ctx->keys[ctx->sorted], ctx->d_count, ctx->ranges, (uint32_t)ntiles,
                                       stats);
    if (ctx->tile_order) {
        k_tile_order<<<1, 1024, 0, st>>>(ctx->ranges, ntiles, ctx->tile_order);
        ++launches;
    }
    GS2_COUNT_LAUNCH(launches + 3);
    return cudaGetLastError();
}
