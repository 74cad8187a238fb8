// Device-wide exclusive scan and stable LSD radix sort used by the tile
// binning of the rasterizer: a depth sort of the Gaussians followed by a
// stable sort of the emitted (tile, Gaussian) pairs by tile id, which
// together order every tile's list by (view depth, Gaussian index).
//
// Radix sort: 8- or 9-bit digits, three kernels per pass over a fixed grid of
// `blocks` CTAs, each owning a contiguous range of the input:
//   hist    per-CTA digit counts (per-warp shared-memory atomics),
//           stored digit-major so that one exclusive scan yields the stable
//           scatter base of every (digit, CTA);
//   scan    one CTA per digit scans its `blocks` counts;
//   scatter each CTA ranks its keys in 2048-key tiles (equal digits found by
//           warp ballots, per-warp digit counters), then writes keys and
//           values to their slots.
// The element count may live on the device (the pair count is only known
// after the binning scan), so no host round trip is needed.
//
// The depth sort, whose count the host knows, takes a one-sweep form of the
// same passes (below): one launch per pass instead of three.
#include "gsc_internal.cuh"

namespace gsc {

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t read_count(const uint32_t* n_dev, uint32_t n_host) {
    if (!n_dev) return n_host;
    uint32_t n = *n_dev;
    return n < n_host ? n : n_host;
}

// contiguous range of CTA b: multiples of the tile so that only the last CTA
// with work has a partial tile
__device__ __forceinline__ void block_range(uint32_t n, int blocks, int b, uint32_t& lo, uint32_t& hi) {
    uint64_t per = ((uint64_t)n + blocks - 1) / blocks;
    per = (per + kSortTile - 1) / kSortTile * kSortTile;
    uint64_t l = per * (uint64_t)b, h = l + per;
    lo = (uint32_t)(l < n ? l : n);
    hi = (uint32_t)(h < n ? h : n);
}

// exclusive scan over a 256-thread block; returns the total in *total
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t v, uint32_t* smem8, uint32_t* total) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem8[warp] = x;
    __syncthreads();
    uint32_t wsum = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        uint32_t s = smem8[w];
        if (w < warp) wsum += s;
        tot += s;
    }
    __syncthreads();
    *total = tot;
    return wsum + x - v;
}

// ------------------------------------------------------------------ radix
//
// DB-bit digits (8 or 9): NDIG = 2^DB buckets.  Per-warp counters keep the
// ranks stable (warps in order, lanes in order within a warp).

template <int DB>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                             const uint32_t* n_dev, uint32_t n_host, int shift,
                                                             uint32_t* __restrict__ hist, int blocks) {
    constexpr int NDIG = 1 << DB;
    __shared__ uint32_t h[8][NDIG];
    uint32_t n = read_count(n_dev, n_host);
    uint32_t lo, hi;
    block_range(n, blocks, blockIdx.x, lo, hi);
    int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 8 * NDIG; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    // 2048 keys per step; the next step's keys are loaded before this
    // step's counts, so one load latency overlaps one step of atomics
    uint32_t kc[kSortIPT];
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
        uint32_t i = lo + j * kSortThreads + threadIdx.x;
        kc[j] = i < hi ? keys[i] : 0u;
    }
    for (uint32_t base = lo; base < hi; base += kSortTile) {
        uint32_t kn[kSortIPT];
        const uint32_t nb = base + kSortTile;
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            uint32_t i = nb + j * kSortThreads + threadIdx.x;
            kn[j] = i < hi ? keys[i] : 0u;
        }
        // plain shared atomics: measured 1.5x faster over the whole pass than
        // aggregating equal digits with __match_any_sync first
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            uint32_t i = base + j * kSortThreads + threadIdx.x;
            if (i < hi) atomicAdd(&h[warp][(kc[j] >> shift) & (uint32_t)(NDIG - 1)], 1u);
            kc[j] = kn[j];
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < NDIG; d += kSortThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += h[w][d];
        hist[(size_t)d * blocks + blockIdx.x] = s;
    }
}

// one CTA per digit: exclusive scan of its per-CTA counts, digit total to totals[d]
__global__ void __launch_bounds__(kSortThreads) k_radix_scan(uint32_t* __restrict__ hist, int blocks,
                                                             uint32_t* __restrict__ totals) {
    __shared__ uint32_t sm[8];
    int d = blockIdx.x;
    uint32_t run = 0;
    for (int b0 = 0; b0 < blocks; b0 += kSortThreads) {
        int b = b0 + threadIdx.x;
        uint32_t v = b < blocks ? hist[(size_t)d * blocks + b] : 0;
        uint32_t tot;
        uint32_t ex = block_exclusive_scan_256(v, sm, &tot);
        if (b < blocks) hist[(size_t)d * blocks + b] = run + ex;
        run += tot;
    }
    if (threadIdx.x == 0) totals[d] = run;
}

// exclusive scan over NDIG per-digit values held DPT = NDIG / 256 per thread
// (thread t owns digits DPT t .. DPT t + DPT - 1)
template <int DPT>
__device__ __forceinline__ void digit_scan(const uint32_t (&v)[DPT], uint32_t (&ex)[DPT], uint32_t* sm) {
    uint32_t t = 0;
#pragma unroll
    for (int k = 0; k < DPT; ++k) t += v[k];
    uint32_t tot;
    uint32_t run = block_exclusive_scan_256(t, sm, &tot);
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
        ex[k] = run;
        run += v[k];
    }
}

template <int DB>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                                const uint32_t* __restrict__ vin,
                                                                uint32_t* __restrict__ kout,
                                                                uint32_t* __restrict__ vout, const uint32_t* n_dev,
                                                                uint32_t n_host, int shift,
                                                                const uint32_t* __restrict__ hist,
                                                                const uint32_t* __restrict__ totals, int blocks) {
    constexpr int NDIG = 1 << DB;
    constexpr int DPT = NDIG / kSortThreads;
    __shared__ uint32_t wh[8][NDIG];
    __shared__ uint32_t dbase[NDIG];
    __shared__ uint32_t tstart[NDIG];
    __shared__ uint32_t gbase[NDIG];
    __shared__ uint32_t skey[kSortTile];
    __shared__ uint32_t sval[kSortTile];
    __shared__ uint32_t sm[8];
    uint32_t n = read_count(n_dev, n_host);
    uint32_t lo, hi;
    block_range(n, blocks, blockIdx.x, lo, hi);
    if (lo >= hi) return;  // uniform per CTA
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        // start of digit d = sum of all smaller digits' totals, plus this CTA's offset within d
        uint32_t v[DPT], ex[DPT];
#pragma unroll
        for (int k = 0; k < DPT; ++k) v[k] = totals[DPT * threadIdx.x + k];
        digit_scan<DPT>(v, ex, sm);
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
            int d = DPT * threadIdx.x + k;
            dbase[d] = ex[k] + hist[(size_t)d * blocks + blockIdx.x];
        }
    }
    unsigned lt = lanemask_lt();
    // keys and values of a tile are loaded one tile ahead: the next tile's
    // loads are issued once this tile sits in shared memory, before its
    // write-out
    uint32_t kk[kSortIPT], vv[kSortIPT];
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
        uint32_t i = lo + warp * (kWarp * kSortIPT) + j * kWarp + lane;
        bool valid = i < hi;
        kk[j] = valid ? kin[i] : 0u;
        vv[j] = valid ? vin[i] : 0u;
    }
    for (uint32_t tile = lo; tile < hi; tile += kSortTile) {
        for (int i = threadIdx.x; i < 8 * NDIG; i += kSortThreads) (&wh[0][0])[i] = 0;
        __syncthreads();
        uint32_t rank[kSortIPT];
        int dd[kSortIPT];
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            uint32_t i = tile + warp * (kWarp * kSortIPT) + j * kWarp + lane;
            bool valid = i < hi;
            int d = valid ? (int)((kk[j] >> shift) & (uint32_t)(NDIG - 1)) : NDIG;
            // lanes with the same digit (NDIG marks an empty slot): one ballot
            // per digit bit, cheaper here than __match_any_sync
            unsigned peers = kFull;
#pragma unroll
            for (int bit = 0; bit <= DB; ++bit) {
                const bool set = (d >> bit) & 1;
                const unsigned m = __ballot_sync(kFull, set);
                peers &= set ? m : ~m;
            }
            uint32_t base = valid ? wh[warp][d] : 0u;
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) wh[warp][d] = base + (uint32_t)__popc(peers);
            __syncwarp();
            rank[j] = base + (uint32_t)__popc(peers & lt);
            dd[j] = d;
        }
        __syncthreads();
        {
            // per digit: warps' offsets within the tile's run of that digit, the
            // run's start in the tile's locally sorted order, and the global
            // position of local element e of digit d (gbase[d] + e)
            uint32_t run[DPT], ts[DPT];
#pragma unroll
            for (int k = 0; k < DPT; ++k) {
                int d = DPT * threadIdx.x + k;
                uint32_t r = 0;
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    uint32_t c = wh[w][d];
                    wh[w][d] = r;
                    r += c;
                }
                run[k] = r;
            }
            digit_scan<DPT>(run, ts, sm);
#pragma unroll
            for (int k = 0; k < DPT; ++k) {
                int d = DPT * threadIdx.x + k;
                tstart[d] = ts[k];
                gbase[d] = dbase[d] - ts[k];
                dbase[d] += run[k];
            }
        }
        __syncthreads();
        // local sort of the tile in shared memory (stable: warp order, then rank)
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            if (dd[j] < NDIG) {
                uint32_t lp = tstart[dd[j]] + wh[warp][dd[j]] + rank[j];
                skey[lp] = kk[j];
                sval[lp] = vv[j];
            }
        }
        const uint32_t nt = tile + kSortTile;
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            uint32_t i = nt + warp * (kWarp * kSortIPT) + j * kWarp + lane;
            bool valid = i < hi;
            kk[j] = valid ? kin[i] : 0u;
            vv[j] = valid ? vin[i] : 0u;
        }
        __syncthreads();
        // runs of equal digits are contiguous in the output: coalesced stores
        const uint32_t cnt = min((uint32_t)kSortTile, hi - tile);
        for (uint32_t e = threadIdx.x; e < cnt; e += kSortThreads) {
            uint32_t k = skey[e];
            uint32_t pos = gbase[(k >> shift) & (uint32_t)(NDIG - 1)] + e;
            kout[pos] = k;
            vout[pos] = sval[e];
        }
        __syncthreads();
    }
}

int sort_blocks_for(uint64_t n) {
    uint64_t b = (n + kSortTile - 1) / kSortTile;
    if (b < 1) b = 1;
    if (b > (uint64_t)kMaxSortBlocks) b = kMaxSortBlocks;
    return (int)b;
}

// CTAs of the scatter kernel that are resident on the device at once: a pass
// runs on at most that many, so that it ends in one wave (a second, partial
// wave would take as long as the first)
template <int DB>
static int resident_scatter_blocks() {
    static int cached = 0;
    if (cached <= 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_radix_scatter<DB>, kSortThreads, 0);
        cached = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
    }
    return cached;
}

// passes = ceil(bits / 9); 8-bit digits when they cover the bits in that
// many passes, else 9-bit digits (e.g. 9 bits: one 9-bit pass; 16: two 8-bit)
int radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const uint32_t* n_dev,
                     uint32_t n_host, int bits, int blocks, uint32_t* hist, cudaStream_t s) {
    uint32_t* totals = radix_totals(hist);
    const int passes = (bits + kMaxDigitBits - 1) / kMaxDigitBits;
    const int db = 8 * passes >= bits ? 8 : 9;
    const int resident = db == 8 ? resident_scatter_blocks<8>() : resident_scatter_blocks<9>();
    if (blocks > resident) blocks = resident;
    int cur = 0;
    for (int shift = 0; shift < bits; shift += db) {
        uint32_t* ki = cur ? k1 : k0;
        uint32_t* vi = cur ? v1 : v0;
        uint32_t* ko = cur ? k0 : k1;
        uint32_t* vo = cur ? v0 : v1;
        if (db == 8) {
            k_radix_hist<8><<<blocks, kSortThreads, 0, s>>>(ki, n_dev, n_host, shift, hist, blocks);
            k_radix_scan<<<256, kSortThreads, 0, s>>>(hist, blocks, totals);
            k_radix_scatter<8><<<blocks, kSortThreads, 0, s>>>(ki, vi, ko, vo, n_dev, n_host, shift, hist, totals,
                                                              blocks);
        } else {
            k_radix_hist<9><<<blocks, kSortThreads, 0, s>>>(ki, n_dev, n_host, shift, hist, blocks);
            k_radix_scan<<<512, kSortThreads, 0, s>>>(hist, blocks, totals);
            k_radix_scatter<9><<<blocks, kSortThreads, 0, s>>>(ki, vi, ko, vo, n_dev, n_host, shift, hist, totals,
                                                              blocks);
        }
        cur ^= 1;
    }
    return cur;
}

int radix_passes(int bits) { return (bits + kMaxDigitBits - 1) / kMaxDigitBits; }

// ------------------------------------------------------------------ one sweep
//
// The depth sort (a count known on the host, 32-bit keys) in 1 + 4 launches
// instead of 3 per pass.  k_os_hist counts the digits of all four 8-bit
// passes in one read of the keys; each pass is then one launch of
// k_os_pass, whose CTAs take the 2048-key tiles in order from a counter.  A
// CTA ranks its tile as k_radix_scatter does, publishes per digit the
// tile's count, and adds the counts of the earlier tiles from the words they
// published (decoupled look-back, Merrill and Garland 2016): a word holds a
// flag and either the tile's own count or the count up to and through that
// tile, and the look-back walks back until it meets the latter.  A key's
// position is the start of its digit over the whole input, plus the digit's
// count in the earlier tiles, plus its rank in the tile, as in the
// three-kernel pass.
//
// Progress: a CTA waits only for tiles taken before its own, whose CTAs are
// already running and publish their count before they wait themselves, so
// every wait ends.  Each is bounded all the same: one that runs out sets
// GSC_ERR_TIMEOUT in the workspace status, and no store of the pass leaves
// the output, whatever the positions.
//
// Scratch (words): digit totals [pass][256], tile counters [pass], then per
// pass one published word per (tile, digit); zeroed before every sort.
constexpr int kOsPasses = 4;
constexpr int kOsDigits = 256;
constexpr size_t kOsHeader = kOsPasses * kOsDigits + 32;
constexpr uint32_t kOsAgg = 1u << 30;  // flag: the tile's own count
constexpr uint32_t kOsInc = 2u << 30;  // flag: the count through the tile
constexpr uint32_t kOsValue = kOsAgg - 1u;
constexpr uint32_t kOsSpinLimit = 1u << 22;
constexpr int kOsWindow = 8;             // predecessors' words loaded at once
constexpr uint32_t kOsHistBlocks = 2 * 152;

size_t onesweep_words(uint64_t n) {
    const uint64_t tiles = (n + kSortTile - 1) / kSortTile;
    return kOsHeader + (size_t)kOsPasses * tiles * kOsDigits;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// digit totals of every pass: per-warp shared counters, then one global
// atomic per (pass, digit) and CTA
__global__ void __launch_bounds__(kSortThreads) k_os_hist(const uint32_t* __restrict__ keys, uint32_t n,
                                                          uint32_t* __restrict__ totals) {
    __shared__ uint32_t h[8][kOsPasses][kOsDigits];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 8 * kOsPasses * kOsDigits; i += kSortThreads) (&h[0][0][0])[i] = 0;
    __syncthreads();
    const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        uint32_t k[kSortIPT];
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            const uint32_t i = t * kSortTile + j * kSortThreads + threadIdx.x;
            k[j] = i < n ? keys[i] : 0u;
        }
#pragma unroll
        for (int j = 0; j < kSortIPT; ++j) {
            if (t * kSortTile + j * kSortThreads + threadIdx.x < n) {
#pragma unroll
                for (int p = 0; p < kOsPasses; ++p) atomicAdd(&h[warp][p][(k[j] >> (8 * p)) & 255u], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kOsPasses * kOsDigits; i += kSortThreads) {
        uint32_t s = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += (&h[w][0][0])[i];
        if (s) atomicAdd(&totals[i], s);
    }
}

// one pass over the 8-bit digit `pass`; one CTA per tile (grid = tiles)
__global__ void __launch_bounds__(kSortThreads) k_os_pass(const uint32_t* __restrict__ kin,
                                                          const uint32_t* __restrict__ vin,
                                                          uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                          uint32_t n, int pass, uint32_t* __restrict__ scratch,
                                                          int32_t* __restrict__ status) {
    __shared__ uint32_t wh[8][kOsDigits];
    __shared__ uint32_t tstart[kOsDigits];
    __shared__ uint32_t gbase[kOsDigits];
    __shared__ uint32_t skey[kSortTile];
    __shared__ uint32_t sval[kSortTile];
    __shared__ uint32_t sm[8];
    __shared__ uint32_t s_tile;
    const int shift = 8 * pass;
    const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
    uint32_t* const word = scratch + kOsHeader + (size_t)pass * tiles * kOsDigits;
    if (threadIdx.x == 0) s_tile = atomicAdd(&scratch[kOsPasses * kOsDigits + pass], 1u);
    for (int i = threadIdx.x; i < 8 * kOsDigits; i += kSortThreads) (&wh[0][0])[i] = 0;
    __syncthreads();
    const uint32_t t = s_tile;  // below tiles: one CTA per tile
    const uint32_t lo = t * kSortTile, hi = min(lo + (uint32_t)kSortTile, n);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    uint32_t kk[kSortIPT], vv[kSortIPT], rank[kSortIPT];
    int dd[kSortIPT];
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
        const uint32_t i = lo + warp * (kWarp * kSortIPT) + j * kWarp + lane;
        const bool valid = i < hi;
        kk[j] = valid ? kin[i] : 0u;
        vv[j] = valid ? vin[i] : 0u;
    }
    // ranks within the tile, stable (warps in order, lanes in order); the
    // digit kOsDigits marks an empty slot
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
        const bool valid = lo + warp * (kWarp * kSortIPT) + j * kWarp + lane < hi;
        const int d = valid ? (int)((kk[j] >> shift) & 255u) : kOsDigits;
        unsigned peers = kFull;
#pragma unroll
        for (int bit = 0; bit <= 8; ++bit) {
            const bool set = (d >> bit) & 1;
            const unsigned m = __ballot_sync(kFull, set);
            peers &= set ? m : ~m;
        }
        const uint32_t base = valid ? wh[warp][d] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wh[warp][d] = base + (uint32_t)__popc(peers);
        __syncwarp();
        rank[j] = base + (uint32_t)__popc(peers & lt);
        dd[j] = d;
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // one digit per thread
        uint32_t r = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const uint32_t c = wh[w][d];
            wh[w][d] = r;
            r += c;
        }
        uint32_t* const mine = word + (size_t)t * kOsDigits + d;
        st_relaxed(mine, (t == 0 ? kOsInc : kOsAgg) | r);
        const uint32_t run[1] = {r}, tot[1] = {scratch[pass * kOsDigits + d]};
        uint32_t ts[1], gs[1];
        digit_scan<1>(run, ts, sm);  // the digit's start in the tile's sorted order
        digit_scan<1>(tot, gs, sm);  // and in the whole output
        // look-back: the digit's count in the tiles before this one, the
        // words of kOsWindow predecessors loaded at once
        uint32_t before = 0;
        bool ok = true, done = t == 0;
        for (uint32_t k = t; !done;) {
            const uint32_t m = k < kOsWindow ? k : kOsWindow;
            uint32_t v[kOsWindow];
#pragma unroll
            for (int i = 0; i < kOsWindow; ++i)
                v[i] = (uint32_t)i < m ? ld_relaxed(word + (size_t)(k - 1 - i) * kOsDigits + d) : 0u;
#pragma unroll
            for (int i = 0; i < kOsWindow; ++i) {
                if (done || (uint32_t)i >= m) break;
                const uint32_t* const w = word + (size_t)(k - 1 - i) * kOsDigits + d;
                for (uint32_t it = 0; (v[i] >> 30) == 0u; v[i] = ld_relaxed(w)) {
                    if (++it == kOsSpinLimit) {
                        ok = false;
                        break;
                    }
                    __nanosleep(64);
                }
                if (!ok) break;
                before += v[i] & kOsValue;
                done = (v[i] & ~kOsValue) == kOsInc;
            }
            k -= m;
            done = done || !ok || k == 0;
        }
        if (t > 0) st_relaxed(mine, kOsInc | ((before + r) & kOsValue));
        if (!ok) atomicCAS(&status[kStatusCode], 0, (int32_t)GSC_ERR_TIMEOUT);
        tstart[d] = ts[0];
        gbase[d] = gs[0] + before - ts[0];
    }
    __syncthreads();
    // local sort of the tile in shared memory, then the runs of equal
    // digits (contiguous in the output) with coalesced stores
#pragma unroll
    for (int j = 0; j < kSortIPT; ++j) {
        if (dd[j] < kOsDigits) {
            const uint32_t lp = tstart[dd[j]] + wh[warp][dd[j]] + rank[j];
            skey[lp] = kk[j];
            sval[lp] = vv[j];
        }
    }
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < hi - lo; e += kSortThreads) {
        const uint32_t k = skey[e];
        const uint32_t pos = gbase[(k >> shift) & 255u] + e;
        if (pos < n) {
            kout[pos] = k;
            vout[pos] = sval[e];
        }
    }
}

int radix_sort_onesweep(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, uint32_t n, uint32_t* scratch,
                        int32_t* status, cudaStream_t s) {
    if (n == 0) return 0;
    const uint32_t tiles = (n + kSortTile - 1) / kSortTile;
    cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * onesweep_words(n), s);
    k_os_hist<<<tiles < kOsHistBlocks ? tiles : kOsHistBlocks, kSortThreads, 0, s>>>(k0, n, scratch);
    int cur = 0;
    for (int p = 0; p < kOsPasses; ++p) {
        k_os_pass<<<tiles, kSortThreads, 0, s>>>(cur ? k1 : k0, cur ? v1 : v0, cur ? k0 : k1, cur ? v0 : v1, n, p,
                                                 scratch, status);
        cur ^= 1;
    }
    return cur;
}

// ------------------------------------------------------------------ scan

// per 2048-item tile sum of cnt[idx[i]]
__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t* __restrict__ cnt,
                                                     const uint32_t* __restrict__ idx, uint32_t n,
                                                     uint32_t* __restrict__ sums) {
    __shared__ uint32_t sm[8];
    uint32_t base = blockIdx.x * kScanTile;
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t i = base + j * 256 + threadIdx.x;
        if (i < n) acc += cnt[idx[i]];
    }
    uint32_t tot;
    block_exclusive_scan_256(acc, sm, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// single CTA: exclusive scan of the tile sums; grand total -> counters, with
// the capacity check of the pair buffers
__global__ void __launch_bounds__(256) k_scan_sums(uint32_t* __restrict__ sums, uint32_t nb,
                                                   uint32_t* __restrict__ counters, int32_t* __restrict__ status,
                                                   uint32_t capacity, unsigned long long* __restrict__ stats) {
    __shared__ uint32_t sm[8];
    uint64_t run = 0;
    for (uint32_t b0 = 0; b0 < nb; b0 += 256) {
        uint32_t b = b0 + threadIdx.x;
        uint32_t v = b < nb ? sums[b] : 0;
        uint32_t tot;
        uint32_t ex = block_exclusive_scan_256(v, sm, &tot);
        if (b < nb) sums[b] = (uint32_t)run + ex;
        run += tot;
    }
    if (threadIdx.x == 0) {
        uint32_t total = run > 0xffffffffull ? 0xffffffffu : (uint32_t)run;
        atomicMax(&counters[kCntPairsMax], total);
        stats[kStPairsSum] += run > capacity ? 0ull : run;
        stats[kStBinnings] += 1ull;
        if (run > capacity) {
            status[kStatusCode] = GSC_ERR_CAPACITY;
            counters[kCntPairs] = 0;  // every later stage of this render does nothing
        } else {
            counters[kCntPairs] = total;
        }
    }
}

__global__ void __launch_bounds__(256) k_scan_apply(const uint32_t* __restrict__ cnt,
                                                    const uint32_t* __restrict__ idx, uint32_t n,
                                                    const uint32_t* __restrict__ sums, uint32_t* __restrict__ out) {
    __shared__ uint32_t sm[8];
    uint32_t base = blockIdx.x * kScanTile;
    uint32_t v[8];
    uint32_t acc = 0;
    // blocked arrangement: thread t owns items base + 8t .. base + 8t + 7
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t i = base + threadIdx.x * 8 + j;
        v[j] = i < n ? cnt[idx[i]] : 0u;
        acc += v[j];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan_256(acc, sm, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        uint32_t i = base + threadIdx.x * 8 + j;
        if (i < n) out[i] = run;
        run += v[j];
    }
}

void scan_gathered(const uint32_t* cnt, const uint32_t* idx, uint32_t n, uint32_t* out, uint32_t* sums,
                   uint32_t* counters, int32_t* status, uint32_t capacity, unsigned long long* stats, cudaStream_t s) {
    uint32_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 0) nb = 1;
    k_scan_reduce<<<nb, 256, 0, s>>>(cnt, idx, n, sums);
    k_scan_sums<<<1, 256, 0, s>>>(sums, nb, counters, status, capacity, stats);
    k_scan_apply<<<nb, 256, 0, s>>>(cnt, idx, n, sums, out);
}

}  // namespace gsc
