// All-source hop-distance BFS on 64-source bitsets, fused with the per-node
// distance histogram.
//
// Method: Algorithm 1 needs, for every node i, the multiset of hop distances
// {dist(i, j)} (Section 3.1, hop reading).  In an undirected graph
// dist(s, v) = dist(v, s), so running a BFS from every source s and counting, at
// node v, how many sources reach v at level d gives v's own histogram h_v(d)
// without any cross-node reduction.
//
// Layout: sources are packed 64 to a uint64 word; a chunk of `wn` consecutive
// words is processed at a time.  Node v owns a row of R 16-byte segments
// (2R >= wn words, node-major) in each of two buffers: the row holds the
// sources known to be within the current level of v.  Level l lives in
// buf[l & 1].
//
// Level 1 (set-up): v's row is {v} + N(v) restricted to the chunk, written
// straight from the CSR.
// Levels l >= 2 (pull): a source s first reaches v at level l exactly when s is
// within level l-1 of a neighbour u and not within level l-1 of v:
//     next[v] = (OR_{u in N(v)} vis_{l-1}[u]) & ~vis_{l-1}[v],   vis_l[v] = vis_{l-1}[v] | next[v]
//     hist[l][v] += popcount(next[v])
// Bits that can never become new start set: sources >= n, the padding word of
// an odd-length row, and sources in another connected component than v (they
// never reach v).  So a row is "all ones" exactly when every source that can
// reach v has, and a saturated row never changes again: sat records the level
// at which each (node, tile) saturated and later levels skip it.
//
// Work: items are (node, tile of 32 segments) taken in the graph's order
// (heaviest degree bucket first; sat is indexed in that order).  Items of rows
// with degree >= 127 are heavy: all warps of a block share one, splitting its
// neighbour list.  Other items go one warp each, 4 list positions per counter
// update (8 with change masks): the first pull level lists every light item, and each level appends
// the items it pulled (still open, or saturated just now and owed one copy of
// ones) to the next level's worklist, so late levels touch only what is left.
// A warp reads its positions' sat words with one load per lane and runs the
// items a ballot marks.  Rows of 32 segments or more are split into tiles
// (lane = segment, G = 32); shorter rows are one tile of G = pow2 >= R lanes and
// the warp reads 32/G neighbours at once.  Neighbour ids are read 32 at a time
// with one coalesced load and broadcast by shuffle; each lane keeps min(4, G)
// loads in flight and stops once its segment has found every missing source.
//
// Change masks (sparse graphs with rows of more than 16 segments): while the
// frontier is sparse, a level also records for each (node, tile) which
// segments gained bits, and the next level reads only those segments of its
// neighbours, skipping neighbours whose tile gained nothing.  This is exact:
// vis_{l-2}[u] is within vis_{l-1}[v] for every neighbour u of v (the
// recurrence above), so a segment of u that did not change at level l-1
// cannot add anything to v at level l.  The first level whose predecessor
// found many bits reads (and writes) no masks, and neither do the levels after it.
//
// One persistent cooperative launch runs the set-up and every level of a
// chunk, separated by a grid barrier whose spin is bounded (on expiry the kernel
// records a timeout and returns).  If the histogram runs out of rows the kernel
// stops at a level boundary and the host grows it and relaunches from that
// level.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "qc_device.cuh"
#include "qc_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t ONES = ~0ull;
constexpr int NOT_SAT = 0x7fffffff;
constexpr int WARPS = 8;               // warps per block
// light list positions taken per counter update: four in the plain variant,
// eight in the change-mask one (measured on GB300: eight took dcsbm-16384's launch
// from 0.359 to 0.473 ms, its scanning levels' tails grew, and sbm-262144's solve
// from 76.8 to 74.2 ms, a quarter as many updates of a counter a million items share)
template <bool MASKS>
__host__ __device__ constexpr int grab_of() { return MASKS ? 8 : 4; }
constexpr int LIST_AFTER = 2;          // pull levels of a launch that scan every item
constexpr int TH_WORDS = 256;          // longest chunk row the two-hop set-up builds in shared memory
constexpr int TH_U = 8;                // neighbour-of-neighbour ids each lane has in flight
constexpr int TH_PIPELINE = 16;        // light nodes per warp from which the set-up takes them ahead
using qcdev::ST_DONE;
using qcdev::ST_NEED_ROWS;
using qcdev::ST_TIMEOUT;
using qcdev::global_ns;
using qcdev::grid_barrier;

struct BfsParams {
    int32_t n;
    const int32_t *row_ptr;
    const int32_t *col_idx;
    const int32_t *order;       // nodes, heaviest degree bucket first; order[n] = heavy count
    const int4 *info;           // {node, row start, row end, 0} per order position
    const int32_t *comp;        // component (smallest node id) of each node
    const int32_t *wcomp;       // component shared by a whole source word, or -1
    const int32_t *wmajor;      // component holding most of a word's sources
    const unsigned long long *wmask;   // bits of those sources
    ulonglong2 *buf[2];         // vis_l in buf[l & 1], [n][R]
    uint32_t *fmask[2];         // [n * T] node-major: bit q of (v, t) set if segment 32t + q of
                                // v's row gained bits at level l (fmask[l & 1]); null below 17 segments
    int32_t mask_ratio;         // read only masked segments at level l when level l-1 found fewer than
                                // (64 wn n) / mask_ratio new bits; 0: never
    int32_t R;                  // 16-byte segments per row in this chunk
    int32_t T;                  // tiles per row
    int32_t w0, wn, W;          // chunk = words [w0, w0 + wn) of W
    uint64_t last_mask;         // bits of sources >= n in word W - 1
    int32_t *sat;               // [n * T], indexed by order position * T + tile
    int32_t *hist;              // [rows][n]
    int32_t rows;
    int32_t first_chunk;        // write hist rows 0 and 1
    int32_t start_level;        // 2: fresh chunk, run the level-1 set-up first
    int32_t *level_new;         // [rows]
    unsigned long long *level_bits;   // [rows] new bits found at each level (level 1: set-up bits)
    int32_t *light_ctr;         // [rows] light list positions taken so far at each level
    int32_t *heavy_ctr;         // [rows] block items taken so far at each level
    int32_t *wl[2];             // worklists of light items: level l reads wl[l & 1]
    int32_t *wl_count;          // [rows] length of each level's worklist
    int32_t *status;            // [0] state, [1] highest level reached (the pass that found nothing);
                                // the graph's outcome words, kept across the chunks of one BFS
    unsigned *bar;              // [0] barrier arrivals over the launch
    unsigned long long *stamp;  // [rows] globaltimer when each level's barrier opened (timing only)
    int32_t *pulled;            // [rows] (node, tile) items pulled at each level (timing only, else null)
    const unsigned long long *deg2;   // sum over nodes of degree^2 (the graph's preparation)
    const int32_t *lo, *hi;     // [n]: the chunk's sources in N(u) are col_idx[lo[u] .. hi[u]) (two-hop set-up)
    int64_t nnz;
    int32_t two_hop;            // levels 1 and 2 from the CSR (two_hop_setup): 0 never, 1 sparse graphs, 2 always
};

__device__ __forceinline__ bool seg_full(const ulonglong2 a) { return (a.x & a.y) == ONES; }

// Bits of one chunk word that start set for node v (other components, sources >= n).
__device__ __forceinline__ uint64_t preset_word(const BfsParams &p, int gw, int cv) {
    uint64_t m;
    const int wc = p.wcomp[gw];
    if (wc >= 0) {
        m = (wc == cv) ? 0ull : ONES;
    } else if (p.wmajor[gw] == cv) {
        m = ~p.wmask[gw];             // v is in the word's main component
    } else {
        m = 0ull;
        const int s0 = 64 * gw;
        const int cnt = min(64, p.n - s0);
        for (int b = 0; b < cnt; ++b)
            if (p.comp[s0 + b] != cv) m |= 1ull << b;
    }
    if (gw == p.W - 1) m |= p.last_mask;
    return m;
}

// ---- level 1 -----------------------------------------------------------------------

// Two passes.  Fill: every row segment gets its preset bits, in node-major
// order so the stores stream; sat starts "not saturated" (level 2 finds the rows
// that are already complete); hist rows 0 and 1 are written for the first chunk.
// Bits: one warp per node sets the bits of v and of its neighbours with
// fire-and-forget atomic ORs (only v's own row is touched, so they never
// contend across warps).
__device__ void init_fill(const BfsParams &p) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    ulonglong2 *out = p.buf[1];
    const long long segs = (long long)p.n * p.R;
    for (long long s = tid; s < segs; s += nthreads) {
        const int v = (int)(s / p.R);
        const int q = (int)(s - (long long)v * p.R);
        const int cv = p.comp[v];
        uint64_t w[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 2 * q + h;
            w[h] = (k < p.wn) ? preset_word(p, p.w0 + k, cv) : ONES;
        }
        out[s] = make_ulonglong2(w[0], w[1]);
    }
    for (int i = tid; i < p.n * p.T; i += nthreads) p.sat[i] = NOT_SAT;
    if (p.fmask[1])
        for (int i = tid; i < p.n * p.T; i += nthreads) p.fmask[1][i] = 0u;
    if (p.first_chunk)
        for (int v = tid; v < p.n; v += nthreads) {
            p.hist[v] = 1;
            p.hist[(size_t)p.n + v] = p.row_ptr[v + 1] - p.row_ptr[v];
        }
}

__device__ void init_bits(const BfsParams &p) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    unsigned long long *words = reinterpret_cast<unsigned long long *>(p.buf[1]);
    const int stride = 2 * p.R;
    uint32_t *fm = p.fmask[1];
    int set = 0;
    for (int v = warp; v < p.n; v += nwarps) {
        unsigned long long *row = words + (size_t)v * stride;
        const int beg = p.row_ptr[v], end = p.row_ptr[v + 1];
        for (int e = beg + lane; e <= end; e += 32) {
            const int u = (e == end) ? v : qcdev::checked_id(p.col_idx[e], p.n, qcdev::DBG_BFS);
            const int k = (u >> 6) - p.w0;
            if (k >= 0 && k < p.wn) {
                atomicOr(row + k, 1ull << (u & 63));
                // segment k / 2 = tile k / 64, bit (k / 2) % 32
                if (fm) atomicOr(fm + (size_t)v * p.T + (k >> 6), 1u << ((k >> 1) & 31));
                ++set;
            }
        }
    }
    set = __reduce_add_sync(FULL, set);
    if (lane == 0 && set) atomicAdd(p.level_bits + 1, (unsigned long long)set);
}

// New bits found by the block at the current level.
__shared__ unsigned int block_found;

// ---- levels 1 and 2 together: the two-hop set-up ------------------------------------
//
// A source s is within two hops of v exactly when s is v, a neighbour of v or a
// neighbour of a neighbour, so vis_2[v] can be written from the CSR alone: the
// preset bits, then v and N(v) (that is vis_1[v]), then N(u) for every u in N(v).
// The bits of vis_2[v] outside vis_1[v] are next_2[v], the sources at distance
// exactly 2, counted into hist[2][v].  This reads sum_u deg(u)^2 neighbour ids,
// against the E neighbour rows of wn/2 segments that the first pull level
// gathers, so a launch takes it on sparse graphs (4 sum deg^2 <= wn E) and it
// then replaces the level-1 set-up and the first pull level.  The row is built
// in shared memory with atomic ORs on 32-bit words; a light node is one warp's,
// a heavy node (degree >= 127, the first order[n] positions) the whole block's.
// The emitting warp keeps vis_1[v] in registers, so the count and, with change
// masks, the segments that gained bits at level 2 come from comparing the two.

constexpr int TH_T = TH_WORDS / 64;     // tiles of a row the set-up builds

// Preset bits of v's row in 64-bit words tid, tid + nt, ... (padding words all ones).
__device__ __forceinline__ void th_preset(const BfsParams &p, uint32_t *row, int v, int tid, int nt) {
    const int cv = p.comp[v];
    unsigned long long *row64 = reinterpret_cast<unsigned long long *>(row);
    for (int k = tid; k < 2 * p.R; k += nt) row64[k] = (k < p.wn) ? preset_word(p, p.w0 + k, cv) : ONES;
}

// Sets source u's bit in the row if u is a source of the chunk.
__device__ __forceinline__ void th_set(const BfsParams &p, uint32_t *row, int u) {
    const int b = u - 64 * p.w0;
    if (b >= 0 && b < 64 * p.wn) atomicOr(row + (b >> 5), 1u << (b & 31));
}

// Bits of v and of its neighbours (ids beg + tid, beg + tid + nt, ...; end stands for
// v); id0, when not negative, is the id at beg + tid, already loaded.
__device__ __forceinline__ void th_first(const BfsParams &p, uint32_t *row, int v, int beg, int end, int tid,
                                         int nt, int id0 = -1) {
    for (int e = beg + tid; e <= end; e += nt)
        th_set(p, row, (e == end) ? v
                       : (e == beg + tid && id0 >= 0) ? id0
                                                     : qcdev::checked_id(p.col_idx[e], p.n, qcdev::DBG_BFS));
}

// The row's segments 32 t + lane (t < T) of this warp, for the comparison at the end.
__device__ __forceinline__ void th_capture(const BfsParams &p, const uint32_t *row, ulonglong2 (&r1)[TH_T]) {
    const int lane = threadIdx.x & 31;
    const ulonglong2 *seg = reinterpret_cast<const ulonglong2 *>(row);
#pragma unroll
    for (int t = 0; t < TH_T; ++t) {
        const int s = 32 * t + lane;
        r1[t] = (t < p.T && s < p.R) ? seg[s] : make_ulonglong2(ONES, ONES);
    }
}

// Start and length of the chunk's part of the neighbour list of u (none for u < 0).
__device__ __forceinline__ void th_bounds(const BfsParams &p, int u, int &ub, int &ul) {
    ub = 0;
    ul = 0;
    if (u >= 0) {
        ub = p.lo[u];
        ul = p.hi[u] - ub;
    }
}

// Neighbour id j0 + lane of a list ending at end, or -1 past its end.
__device__ __forceinline__ int th_id(const BfsParams &p, int j0, int end) {
    const int e = j0 + (threadIdx.x & 31);
    return e < end ? qcdev::checked_id(p.col_idx[e], p.n, qcdev::DBG_BFS) : -1;
}

// th_bounds of batch member `lane` (ids j0 + lane).
__device__ __forceinline__ void th_lists(const BfsParams &p, int j0, int end, int &ub, int &ul) {
    th_bounds(p, th_id(p, j0, end), ub, ul);
}

// Bits of the neighbours of v's neighbours, for the neighbour batches of 32 starting
// at beg + 32 sub, stride 32 nsub (one warp of nsub); (ub0, ul0) are the lists of the
// first batch, fetched by the caller.  The batch's lists are laid end to end and the
// warp walks that concatenation 32 ids at a time, each lane finding the list its
// position falls in by a binary search over the batch's exclusive prefix sums.
// Under the selection rule a degree is at most sqrt(wn E / 4) < 2^19 (forced:
// below 2^20), so a batch's total fits an int.
__device__ __forceinline__ void th_second(const BfsParams &p, uint32_t *row, int beg, int end, int sub, int nsub,
                                          int ub, int ul) {
    const int lane = threadIdx.x & 31;
    for (int j0 = beg + 32 * sub; j0 < end; j0 += 32 * nsub) {
        if (j0 != beg + 32 * sub) th_lists(p, j0, end, ub, ul);
        int incl = ul;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += y;
        }
        const int total = __shfl_sync(FULL, incl, 31);
        const int excl = incl - ul;
        for (int f0 = 0; f0 < total; f0 += 32 * TH_U) {
            int w[TH_U];
#pragma unroll
            for (int k = 0; k < TH_U; ++k) {
                const int f = f0 + 32 * k + lane;
                // the last lane i with excl_i <= f owns position f (lists of length 0
                // share their successor's start, so the last one wins)
                int i = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (__shfl_sync(FULL, excl, i + step) <= f) i += step;
                const int at = __shfl_sync(FULL, ub, i) + (f - __shfl_sync(FULL, excl, i));
                w[k] = (f < total) ? qcdev::checked_id(p.col_idx[at], p.n, qcdev::DBG_BFS) : -1;
            }
#pragma unroll
            for (int k = 0; k < TH_U; ++k)
                if (w[k] >= 0) th_set(p, row, w[k]);
        }
    }
}

// One warp writes the finished row of v (order position oi) as level 2, its tiles'
// saturation (level 2 if all ones) and change masks, and v's histogram entries.
template <bool MASKS>
__device__ __forceinline__ bool th_emit(const BfsParams &p, const uint32_t *row, const ulonglong2 (&r1)[TH_T], int v,
                                        int oi, int deg) {
    const int lane = threadIdx.x & 31;
    const ulonglong2 *seg = reinterpret_cast<const ulonglong2 *>(row);
    ulonglong2 *out = p.buf[0] + (size_t)v * p.R;
    int count = 0;
    unsigned fulls = 0u, chgs[TH_T];
#pragma unroll
    for (int t = 0; t < TH_T; ++t) {
        const int s = 32 * t + lane;
        bool full = true, changed = false;
        if (t < p.T && s < p.R) {
            const ulonglong2 x = seg[s];
            out[s] = x;
            full = seg_full(x);
            count += __popcll(x.x & ~r1[t].x) + __popcll(x.y & ~r1[t].y);
            changed = x.x != r1[t].x || x.y != r1[t].y;
        }
        if (__all_sync(FULL, full)) fulls |= 1u << t;
        chgs[t] = __ballot_sync(FULL, changed);
    }
    if (lane < p.T) {
        const int t = lane;
        p.sat[(size_t)oi * p.T + t] = ((fulls >> t) & 1u) ? 2 : NOT_SAT;
        if constexpr (MASKS) {
            unsigned c = chgs[0];
#pragma unroll
            for (int k = 1; k < TH_T; ++k)
                if (t == k) c = chgs[k];
            p.fmask[0][(size_t)v * p.T + t] = c;
            p.fmask[1][(size_t)v * p.T + t] = 0u;
        }
    }
    count = __reduce_add_sync(FULL, count);
    if (lane == 0) {
        if (p.first_chunk) {
            p.hist[v] = 1;
            p.hist[(size_t)p.n + v] = deg;
        }
        if (count) p.hist[2 * (size_t)p.n + v] += count;
        if constexpr (MASKS) {
            if (count) atomicAdd(&block_found, (unsigned)count);
        }
    }
    return count != 0;
}

// Levels 1 and 2 of a chunk: heavy nodes block by block, then light nodes warp by
// warp, both taken from counters.  rows: WARPS rows of 2 TH_WORDS 32-bit words.
// Returns whether this thread's rows gained bits at level 2.
template <bool MASKS>
__device__ __forceinline__ bool two_hop_setup(const BfsParams &p, uint32_t (*rows)[2 * TH_WORDS]) {
    bool any_new = false;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int heavy = p.order[p.n];
    __shared__ int th_grab;
    ulonglong2 r1[TH_T];
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) th_grab = atomicAdd(p.heavy_ctr + 1, 1);
        __syncthreads();
        const int oi = th_grab;
        if (oi >= heavy) break;
        const int4 inf = p.info[oi];
        uint32_t *row = rows[0];
        int ub, ul;
        th_lists(p, inf.y + 32 * wib, inf.z, ub, ul);
        th_preset(p, row, inf.x, threadIdx.x, blockDim.x);
        __syncthreads();
        th_first(p, row, inf.x, inf.y, inf.z, threadIdx.x, blockDim.x);
        __syncthreads();
        if (wib == 0) th_capture(p, row, r1);
        __syncthreads();
        th_second(p, row, inf.y, inf.z, wib, WARPS, ub, ul);
        __syncthreads();
        if (wib == 0 && th_emit<MASKS>(p, row, r1, inf.x, oi, inf.z - inf.y)) any_new = true;
    }
    uint32_t *row = rows[wib];
    if (p.n - heavy < TH_PIPELINE * ((gridDim.x * blockDim.x) >> 5)) {
        // few nodes per warp: take one at a time, so the last ones go to idle warps
        while (true) {
            int oi = 0;
            if (lane == 0) oi = heavy + atomicAdd(p.light_ctr + 1, 1);
            oi = __shfl_sync(FULL, oi, 0);
            if (oi >= p.n) break;
            const int4 inf = p.info[oi];
            const int id = th_id(p, inf.y, inf.z);
            int ub, ul;
            th_bounds(p, id, ub, ul);
            th_preset(p, row, inf.x, lane, 32);
            __syncwarp();
            th_first(p, row, inf.x, inf.y, inf.z, lane, 32, id);
            __syncwarp();
            th_capture(p, row, r1);
            th_second(p, row, inf.y, inf.z, 0, 1, ub, ul);
            __syncwarp();
            if (th_emit<MASKS>(p, row, r1, inf.x, oi, inf.z - inf.y)) any_new = true;
            __syncwarp();
        }
        return any_new;
    }
    // many nodes per warp: pipelined, so while node k is built the warp already holds
    // node k+1's position, row bounds and first neighbour ids, and node k+2's position
    // is on its way
    const int4 none = make_int4(0, 0, 0, 0);
    int ahead = 0;
    if (lane == 0) ahead = heavy + atomicAdd(p.light_ctr + 1, 1);
    int oi = __shfl_sync(FULL, ahead, 0);
    int4 inf = oi < p.n ? p.info[oi] : none;
    int id = oi < p.n ? th_id(p, inf.y, inf.z) : -1;
    if (lane == 0) ahead = heavy + atomicAdd(p.light_ctr + 1, 1);
    while (oi < p.n) {
        const int oi1 = __shfl_sync(FULL, ahead, 0);
        const int4 inf1 = oi1 < p.n ? p.info[oi1] : none;
        if (lane == 0) ahead = heavy + atomicAdd(p.light_ctr + 1, 1);
        int ub, ul;
        th_bounds(p, id, ub, ul);
        th_preset(p, row, inf.x, lane, 32);
        __syncwarp();
        th_first(p, row, inf.x, inf.y, inf.z, lane, 32, id);
        __syncwarp();
        th_capture(p, row, r1);
        th_second(p, row, inf.y, inf.z, 0, 1, ub, ul);
        const int id1 = oi1 < p.n ? th_id(p, inf1.y, inf1.z) : -1;
        __syncwarp();
        if (th_emit<MASKS>(p, row, r1, inf.x, oi, inf.z - inf.y)) any_new = true;
        __syncwarp();
        oi = oi1;
        inf = inf1;
        id = id1;
    }
    return any_new;
}

// hi[u] = the first position of N(u) at or after lo[u] whose id is >= bound (rows
// are sorted): with lo at the chunk's first source, [lo[u], hi[u]) is N(u)
// restricted to the chunk, and hi is the next chunk's lo.
__global__ void chunk_cursor(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *lo,
                             int32_t bound, int32_t *hi) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        int a = lo[u], b = row_ptr[u + 1];
        while (a < b) {
            const int m = a + ((b - a) >> 1);
            if (col_idx[m] < bound) a = m + 1;
            else b = m;
        }
        hi[u] = a;
    }
}

// Whether a fresh chunk's levels 1 and 2 come from the two-hop set-up (the same
// answer in bfs_two_hop and bfs_persistent).  two_hop 1: on sparse graphs; 2: on
// every graph whose degrees are below 2^20 (their squares sum below 2^40), which
// keeps a batch's id count within an int.
__device__ __forceinline__ bool two_hop_taken(const BfsParams &p) {
    if (p.start_level != 2 || p.rows <= 2 || 2 * p.R > TH_WORDS) return false;
    const unsigned long long d2 = *p.deg2;
    return (p.two_hop == 1 && 4ull * d2 <= (unsigned long long)p.wn * (unsigned long long)p.nnz) ||
           (p.two_hop == 2 && d2 < (1ull << 40));
}

// The two-hop set-up as its own launch, queued just before bfs_persistent: levels
// 1 and 2 of the chunk, hist rows 0-2, the items' saturation, level 2's flag and
// (with masks) its change masks and bit count.
template <bool MASKS>
__global__ void __launch_bounds__(256) bfs_two_hop(const BfsParams p) {
    __shared__ __align__(16) uint32_t rows[WARPS][2 * TH_WORDS];
    if (!two_hop_taken(p)) return;
    if (threadIdx.x == 0) block_found = 0u;
    if (p.stamp && blockIdx.x == 0 && threadIdx.x == 0) p.stamp[1] = global_ns();
    __syncthreads();
    const bool any_new = two_hop_setup<MASKS>(p, rows);
    if (__syncthreads_or(any_new) && threadIdx.x == 0) p.level_new[2] = 1;
    if constexpr (MASKS) {
        // a count past 2^32 in one block only misjudges the density estimate
        if (threadIdx.x == 0 && block_found) atomicAdd(p.level_bits + 2, (unsigned long long)block_found);
    }
}

// ---- levels >= 2: pull ------------------------------------------------------------

// Items the block pulled at the current level (reported in timing mode).
__shared__ unsigned int block_pulled;
// Per warp: ids and change masks of the neighbours a G = 32 gather reads.
__shared__ int2 pack[WARPS][32];

// OR of the rows of neighbours [j_first, end) of one node, taking 32-neighbour
// chunks j_first, j_first + stride, ... (stride = 32 x the warps sharing the row).
// Lane (slot, q) accumulates segment q; it stops once acc | own is all ones.
// When `have0` is set, myu0 already holds the first chunk's ids (prefetched).
// At a masked level (MASKS, G = 32: lane = segment of tile t) only the
// neighbours whose tile changed at the previous level are read, packed (id and
// change mask) into the warp's slots in shared memory, each only in the
// segments whose bit is set: a segment of u that gained nothing at level l-1
// equals u's segment at level l-2, which the recurrence already put into v's
// row at level l-1.
template <int G, bool MASKS>
__device__ __forceinline__ ulonglong2 gather_or(const BfsParams &p, const int level, int j_first, int end,
                                                int stride, int q, bool qok, ulonglong2 own, bool masked, int t,
                                                bool have0 = false, int myu0 = 0) {
    const ulonglong2 *vin = p.buf[(level - 1) & 1];
    constexpr int SLOTS = 32 / G;
    constexpr int U = G < 4 ? G : 4;
    const int lane = threadIdx.x & 31;
    const int slot = lane / G;
    const ulonglong2 zero = make_ulonglong2(0ull, 0ull);
    ulonglong2 acc = zero;
    bool act = !seg_full(own);
    for (int j0 = j_first; j0 < end; j0 += stride) {
        if (!__any_sync(FULL, act)) break;
        const int cnt = min(32, end - j0);
        const int myu = (have0 && j0 == j_first) ? myu0 : ((lane < cnt) ? qcdev::checked_id(p.col_idx[j0 + lane], p.n, qcdev::DBG_BFS) : 0);
        if (G == 32 && MASKS && masked) {
            const uint32_t fm = (lane < cnt) ? p.fmask[(level - 1) & 1][(size_t)myu * p.T + t] : 0u;
            const unsigned nz = __ballot_sync(FULL, fm != 0u);
            const int live = __popc(nz);
            int2 *slots = pack[threadIdx.x >> 5];
            if (fm) slots[__popc(nz & ((1u << lane) - 1u))] = make_int2(myu, (int)fm);
            __syncwarp();
            for (int m = 0; m < live; m += U) {
                ulonglong2 x[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    const int2 e = (m + k < live) ? slots[m + k] : make_int2(0, 0);
                    x[k] = (act && qok && ((e.y >> lane) & 1)) ? vin[(size_t)e.x * p.R + q] : zero;
                }
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    acc.x |= x[k].x;
                    acc.y |= x[k].y;
                }
                act = act && !seg_full(make_ulonglong2(acc.x | own.x, acc.y | own.y));
                if (!__any_sync(FULL, act)) break;
            }
            __syncwarp();
        } else {
            for (int m = 0; m < cnt; m += SLOTS * U) {
                ulonglong2 x[U];
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    const int tt = m + k * SLOTS + slot;
                    const int u = __shfl_sync(FULL, myu, tt & 31);
                    x[k] = (act && qok && tt < cnt) ? vin[(size_t)u * p.R + q] : zero;
                }
#pragma unroll
                for (int k = 0; k < U; ++k) {
                    acc.x |= x[k].x;
                    acc.y |= x[k].y;
                }
                act = act && !seg_full(make_ulonglong2(acc.x | own.x, acc.y | own.y));
                if (!__any_sync(FULL, act)) break;
            }
        }
    }
    return acc;
}


// Finish one item: combine the slots, write the row segment, count, mark
// saturation; at a masked level of a MASKS launch, also record which segments of
// the tile gained bits and add the bits found to the block's count.
template <int G, bool MASKS>
__device__ __forceinline__ void finish_item(const BfsParams &p, ulonglong2 acc, const ulonglong2 own,
                                            ulonglong2 *orow, int q, bool qok, int v, int sidx,
                                            int32_t *hrow, int level, bool masked, bool &any_new) {
    const int lane = threadIdx.x & 31;
    const int slot = lane / G;
#pragma unroll
    for (int off = G; off < 32; off <<= 1) {
        acc.x |= __shfl_xor_sync(FULL, acc.x, off);
        acc.y |= __shfl_xor_sync(FULL, acc.y, off);
    }
    int count = 0;
    bool full = true;
    if (slot == 0 && qok) {
        const ulonglong2 nw = make_ulonglong2(acc.x & ~own.x, acc.y & ~own.y);
        const ulonglong2 o = make_ulonglong2(own.x | nw.x, own.y | nw.y);
        orow[q] = o;
        count = __popcll(nw.x) + __popcll(nw.y);
        full = seg_full(o);
    }
    if constexpr (G == 32 && MASKS) {
        if (masked) {
            const unsigned changed = __ballot_sync(FULL, count != 0);
            if (lane == 0) p.fmask[level & 1][(size_t)v * p.T + (q >> 5)] = changed;
        }
    }
    count = __reduce_add_sync(FULL, count);
    full = __all_sync(FULL, full);
    if (lane == 0) {
        if (count) {
            if (p.T > 1) atomicAdd(hrow + v, count);
            else hrow[v] += count;
            if constexpr (MASKS) {
                if (masked) atomicAdd(&block_found, (unsigned)count);
            }
            any_new = true;
        }
        if (full) p.sat[sidx] = level;
    }
}

// Heavy rows (the first order[n] nodes, rows of 32 segments or more): one block
// per (node, tile) item; warp w takes neighbour chunks w, w + 8, ...; the
// partial ORs meet in shared memory and warp 0 finishes.
template <bool MASKS>
__device__ void heavy_items(const BfsParams &p, const int level, const bool masked, bool &any_new,
                            ulonglong2 (*red)[32]) {
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const ulonglong2 *vin = p.buf[(level - 1) & 1];
    ulonglong2 *vout = p.buf[level & 1];
    int32_t *hrow = p.hist + (size_t)level * p.n;
    const int items = p.order[p.n] * p.T;
    __shared__ int grab;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) grab = atomicAdd(p.heavy_ctr + level, 1);
        __syncthreads();
        const int it = grab;
        if (it >= items) break;
        const int oi = it / p.T;
        const int4 inf = p.info[oi];
        const int sv = p.sat[it];
        if (sv <= level - 2) continue;
        const int t = it - oi * p.T;
        const int v = inf.x;
        const int q = t * 32 + lane;
        const bool qok = q < p.R;
        ulonglong2 *orow = vout + (size_t)v * p.R;
        if (sv == level - 1) {
            if (wib == 0 && qok) orow[q] = make_ulonglong2(ONES, ONES);
            continue;
        }
        if (threadIdx.x == 0) block_pulled += 1u;
        const ulonglong2 own = qok ? vin[(size_t)v * p.R + q] : make_ulonglong2(ONES, ONES);
        const int beg = inf.y, end = inf.z;
        red[wib][lane] = gather_or<32, MASKS>(p, level, beg + 32 * wib, end, 32 * WARPS, q, qok, own, masked, t);
        __syncthreads();
        if (wib == 0) {
            ulonglong2 acc = red[0][lane];
            for (int w = 1; w < WARPS; ++w) {
                acc.x |= red[w][lane].x;
                acc.y |= red[w][lane].y;
            }
            finish_item<32, MASKS>(p, acc, own, orow, q, qok, v, it, hrow, level, masked, any_new);
        }
    }
}

// Light items: a warp takes grab_of<MASKS>() list positions, one sat word per lane, and
// runs the items a ballot marks (copy-ones items first, then pull items); the
// pull items go to the next level's worklist.  The first pull level of a
// launch lists every light item in order; later levels read the worklist.
template <int G, bool MASKS>
__device__ __forceinline__ void light_items(const BfsParams &p, const int level, const bool from_list,
                                            const bool make_list, const bool masked, bool &any_new) {
    const int lane = threadIdx.x & 31;
    const int slot = lane / G;
    const int ql = lane % G;
    const ulonglong2 *vin = p.buf[(level - 1) & 1];
    ulonglong2 *vout = p.buf[level & 1];
    int32_t *hrow = p.hist + (size_t)level * p.n;
    const int first = (G == 32) ? p.order[p.n] * p.T : 0;   // heavy items go to heavy_items
    const int32_t *src = p.wl[level & 1];
    int32_t *dst = p.wl[(level + 1) & 1];
    const int count = from_list ? *(volatile int32_t *)(p.wl_count + level) : p.n * p.T - first;
    int32_t *ctr = p.light_ctr + level;
    int base = 0;
    constexpr int GRAB = grab_of<MASKS>();
    if (lane == 0) base = atomicAdd(ctr, GRAB);
    base = __shfl_sync(FULL, base, 0);
    while (base < count) {
        int next = 0;
        if (lane == 0) next = atomicAdd(ctr, GRAB);
        const int pos = base + lane;
        const bool has = lane < GRAB && pos < count;
        const int it = has ? (from_list ? src[pos] : first + pos) : 0;
        const int oi = it / p.T;
        // the item's saturation level and its node's row come in two independent loads
        const int4 inf = has ? p.info[oi] : make_int4(0, 0, 0, 0);
        const int sv = has ? p.sat[it] : 0;
        const bool ones = has && sv == level - 1;
        const bool pull = has && sv > level - 1;
        const int v_l = inf.x;
        const int t_l = it - oi * p.T;
        const int beg_l = pull ? inf.y : 0;
        const int end_l = pull ? inf.z : 0;
        unsigned mask = __ballot_sync(FULL, ones);
        while (mask) {
            const int b = __ffs(mask) - 1;
            mask &= mask - 1;
            const int v = __shfl_sync(FULL, v_l, b);
            const int t = __shfl_sync(FULL, t_l, b);
            const int q = t * 32 + ql;
            if (slot == 0 && q < p.R) vout[(size_t)v * p.R + q] = make_ulonglong2(ONES, ONES);
        }
        const unsigned pulls = __ballot_sync(FULL, pull);
        // (rows of fewer than 17 segments always fit L2, so only the tiled variant counts)
        if constexpr (G == 32) {
            if (lane == 0 && pulls) atomicAdd(&block_pulled, (unsigned)__popc(pulls));
        }
        mask = pulls;
        if constexpr (MASKS) {
            // item state: the next item's own segment and first neighbour ids are
            // requested before the current item's gathers, so the two overlap; the
            // rest is shuffled again from the lane b that holds it when needed
            struct Item {
                int b, myu;
                ulonglong2 own;
            };
            auto fetch = [&](int b, Item &x) {
                x.b = b;
                const int v = __shfl_sync(FULL, v_l, b);
                const int q = __shfl_sync(FULL, t_l, b) * 32 + ql;
                const int beg = __shfl_sync(FULL, beg_l, b);
                const int len = __shfl_sync(FULL, end_l, b) - beg;
                x.own = (q < p.R) ? vin[(size_t)v * p.R + q] : make_ulonglong2(ONES, ONES);
                x.myu = (lane < len) ? qcdev::checked_id(p.col_idx[beg + lane], p.n, qcdev::DBG_BFS) : 0;
            };
            Item cur, nxt;
            if (mask) fetch(__ffs(mask) - 1, cur);
            while (mask) {
                mask &= mask - 1;
                if (mask) fetch(__ffs(mask) - 1, nxt);
                const int v = __shfl_sync(FULL, v_l, cur.b);
                const int t = __shfl_sync(FULL, t_l, cur.b);
                const int q = t * 32 + ql;
                const bool qok = q < p.R;
                const ulonglong2 acc = gather_or<G, true>(p, level, __shfl_sync(FULL, beg_l, cur.b),
                                                          __shfl_sync(FULL, end_l, cur.b), 32, q, qok, cur.own,
                                                          masked, t, true, cur.myu);
                finish_item<G, true>(p, acc, cur.own, vout + (size_t)v * p.R, q, qok, v,
                                     __shfl_sync(FULL, it, cur.b), hrow, level, masked, any_new);
                cur = nxt;
            }
        } else {
            // item state; the next item's own segment and first neighbour ids are
            // requested before the current item's gathers, so the two overlap
            struct Item {
                int v, t, sidx, beg, end, myu;
                ulonglong2 own;
            };
            auto fetch = [&](int b, Item &x) {
                x.v = __shfl_sync(FULL, v_l, b);
                x.t = __shfl_sync(FULL, t_l, b);
                x.sidx = __shfl_sync(FULL, it, b);
                x.beg = __shfl_sync(FULL, beg_l, b);
                x.end = __shfl_sync(FULL, end_l, b);
                const int q = x.t * 32 + ql;
                x.own = (q < p.R) ? vin[(size_t)x.v * p.R + q] : make_ulonglong2(ONES, ONES);
                x.myu = (lane < x.end - x.beg) ? qcdev::checked_id(p.col_idx[x.beg + lane], p.n, qcdev::DBG_BFS) : 0;
            };
            Item cur, nxt;
            if (mask) fetch(__ffs(mask) - 1, cur);
            while (mask) {
                mask &= mask - 1;
                if (mask) fetch(__ffs(mask) - 1, nxt);
                const int q = cur.t * 32 + ql;
                const bool qok = q < p.R;
                const ulonglong2 acc =
                    gather_or<G, false>(p, level, cur.beg, cur.end, 32, q, qok, cur.own, false, 0, true, cur.myu);
                finish_item<G, false>(p, acc, cur.own, vout + (size_t)cur.v * p.R, q, qok, cur.v, cur.sidx, hrow,
                                      level, masked, any_new);
                cur = nxt;
            }
        }
        if (make_list && pulls) {
            int at = 0;
            if (lane == 0) at = atomicAdd(p.wl_count + level + 1, __popc(pulls));
            at = __shfl_sync(FULL, at, 0);
            if (pull) dst[at + __popc(pulls & ((1u << lane) - 1))] = it;
        }
        base = __shfl_sync(FULL, next, 0);
    }
}

// MASKS: the variant that keeps change masks (G = 32 only), for graphs whose
// early frontiers are sparse; the plain variant reads every segment of every
// neighbour.
// Blocks per SM: four (64 registers) for the short-row variants and the
// change-mask one, three (80 registers) for the plain tiled one.  Measured on
// GB300: four blocks took the plain variant on dcsbm-16384 from 0.359 to 0.412
// ms per launch (its spills), and the mask variant on sbm-262144 from 79.1 to
// 77.6 ms per solve.
template <int G, bool MASKS>
__global__ void __launch_bounds__(256, (G == 32 && !MASKS) ? 3 : 4) bfs_persistent(const BfsParams p) {
    __shared__ ulonglong2 red[WARPS][32];
    if (threadIdx.x == 0) {
        block_found = 0u;
        block_pulled = 0u;
    }
    __syncthreads();
    int level = p.start_level;
    const bool stamp = p.stamp && blockIdx.x == 0 && threadIdx.x == 0;
    const bool after_two_hop = two_hop_taken(p);
    if (stamp && !after_two_hop) p.stamp[level - 1] = global_ns();
    if (level == 2) {
        if (after_two_hop) {
            // bfs_two_hop wrote levels 1 and 2
            if (stamp) p.stamp[2] = p.stamp[3] = global_ns();
            if (*(volatile int32_t *)(p.level_new + 2) == 0) {
                // nothing at distance 2: the BFS ends here
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(p.status + 1, 2);
                return;
            }
            level = 3;
        } else {
            init_fill(p);
            if (!grid_barrier(p.bar, p.status)) return;
            init_bits(p);
            if (!grid_barrier(p.bar, p.status)) return;
            if (stamp) p.stamp[2] = global_ns();
        }
    }
    // masks of the previous level are complete: the set-up writes level 1's, and
    // a masked level writes its own; after the first level that is not masked
    // none are written again (the frontiers only fill up from there), and a
    // relaunch from a later level starts without them
    bool masks_ok = p.start_level == 2;
    for (;; ++level) {
        if (level >= p.rows) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                atomicMax(p.status + 1, level);
                atomicCAS(p.status, ST_DONE, ST_NEED_ROWS);
            }
            return;
        }
        // a MASKS launch reads and writes change masks at this level while the
        // previous one found few bits (most segments unchanged)
        bool masked = false;
        if constexpr (MASKS) {
            masked = masks_ok &&
                     *(volatile unsigned long long *)(p.level_bits + level - 1) * (unsigned long long)p.mask_ratio <
                         64ull * (unsigned long long)p.wn * (unsigned long long)p.n;
            masks_ok = masked;
        }
        bool any_new = false;
        if (G == 32) heavy_items<MASKS>(p, level, masked, any_new, red);
        // the first pull levels touch nearly every item: scan them all; from the
        // third on, each level lists what it pulled for the next
        light_items<G, MASKS>(p, level, level >= p.start_level + LIST_AFTER + 1,
                              level >= p.start_level + LIST_AFTER, masked, any_new);
        if (__syncthreads_or(any_new) && threadIdx.x == 0) p.level_new[level] = 1;
        if (threadIdx.x == 0) {
            if (p.pulled && block_pulled) atomicAdd(p.pulled + level, (int)block_pulled);
            block_pulled = 0u;
        }
        if constexpr (MASKS) {
            // a count past 2^32 in one block only misjudges the density estimate
            if (threadIdx.x == 0) {
                if (block_found) atomicAdd(p.level_bits + level, (unsigned long long)block_found);
                block_found = 0u;
            }
        }
        if (!grid_barrier(p.bar, p.status)) return;
        if (stamp) p.stamp[level + 1] = global_ns();
        if (*(volatile int32_t *)(p.level_new + level) == 0) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicMax(p.status + 1, level);
}

typedef void (*bfs_fn)(const BfsParams);

bfs_fn pick(int R, bool masks, int *G) {
    if (R <= 1) { *G = 1; return bfs_persistent<1, false>; }
    if (R <= 2) { *G = 2; return bfs_persistent<2, false>; }
    if (R <= 4) { *G = 4; return bfs_persistent<4, false>; }
    if (R <= 8) { *G = 8; return bfs_persistent<8, false>; }
    if (R <= 16) { *G = 16; return bfs_persistent<16, false>; }
    *G = 32;
    return masks ? bfs_persistent<32, true> : bfs_persistent<32, false>;
}

// Grow hist to at least `rows` levels (new rows zeroed), keeping the old rows.
qc_status ensure_hist_rows(qc_graph *g, int32_t rows, cudaStream_t stream) {
    if (rows <= g->hist_rows) return QC_OK;
    int32_t want = g->hist_rows ? g->hist_rows : 16;
    while (want < rows) want *= 2;
    if (want > g->n + 1) want = (g->n + 1 > rows) ? g->n + 1 : rows;
    qc_buffer nb;
    const size_t row_bytes = sizeof(int32_t) * (size_t)g->n;
    QC_TRY(nb.allocate(g->ctx, row_bytes * (size_t)want, stream));
    QC_CUDA_TRY(g->ctx, cudaMemsetAsync(nb.ptr, 0, nb.bytes, stream));
    if (g->hist_rows)
        QC_CUDA_TRY(g->ctx, cudaMemcpyAsync(nb.ptr, g->hist.ptr, row_bytes * (size_t)g->hist_rows,
                                            cudaMemcpyDeviceToDevice, stream));
    g->hist = std::move(nb);
    g->hist_rows = want;
    return QC_OK;
}

}  // namespace

// Modelled algorithmic bytes of one level pass over a chunk of wn source words
// (pull over every node): per node and word, gather the row word of each
// neighbour, read the node's own word and write it back, plus one write of the
// next-frontier word (8 wn (E + 3N)); the CSR once (4(N+1) + 4E); one histogram
// row (4N).
double qc_bfs_level_model_bytes(int64_t n, int64_t nnz, int64_t wn) {
    return 8.0 * (double)wn * (double)(nnz + 3 * n) + 4.0 * (double)(n + 1) + 4.0 * (double)nnz +
           4.0 * (double)n;
}

// Scratch of one all-source BFS: chunk width, variant, bitset buffers, item state,
// worklists and the control block.  Sized once per graph and reused by every
// chunk (and, in a captured plan, by every replay).
qc_status qc_bfs_scratch_init(qc_graph *g, qc_bfs_scratch &bs, cudaStream_t stream) {
    qc_ctx *ctx = g->ctx;
    const int32_t n = g->n;
    bs.wc = qc_bfs_chunk_words(ctx, n);
    bs.R_max = (bs.wc + 1) / 2;
    bs.T_max = bs.R_max >= 32 ? (bs.R_max + 31) / 32 : 1;
    const size_t vis_bytes = sizeof(ulonglong2) * (size_t)bs.R_max * (size_t)n;
    QC_TRY(bs.visA.allocate(ctx, vis_bytes, stream));
    QC_TRY(bs.visB.allocate(ctx, vis_bytes, stream));
    // Change masks (rows of more than 16 segments) pay off when the frontiers of the
    // first pull levels are sparse: a tree-like graph of mean degree d reaches about
    // d^2 of its n nodes in two hops, so the variant with masks is taken when
    // d^2 * mask_ratio < n (a level then reads masked segments while the previous
    // level found fewer than 64 wn n / mask_ratio new bits).  Measured on GB300:
    // SBM of mean degree 20 with n = 2^16 and 2^18, 7 % and 11 % faster; a
    // DC-SBM of n = 2^14 and mean degree 16, 5 % slower (only its level 2 is sparse).
    // QCGRAPH_MASK_RATIO overrides the ratio (0: never).
    bs.mask_ratio = 128;
    if (const char *env = getenv("QCGRAPH_MASK_RATIO")) bs.mask_ratio = std::max(0, atoi(env));
    const double mean_deg = (double)g->nnz / (double)n;
    bs.masks = bs.mask_ratio > 0 && bs.R_max > 16 && mean_deg * mean_deg * bs.mask_ratio < (double)n;
    // QCGRAPH_TWO_HOP: 0 keeps the level-1 set-up and the first pull level on every
    // graph, 2 takes the two-hop set-up wherever its row fits (tests), 1 (default)
    // on sparse graphs
    bs.two_hop = 1;
    if (const char *env = getenv("QCGRAPH_TWO_HOP")) bs.two_hop = std::min(2, std::max(0, atoi(env)));
    if (bs.two_hop && bs.wc < (n + 63) / 64 && bs.R_max * 2 <= TH_WORDS)
        QC_TRY(bs.cursor.allocate(ctx, 2 * sizeof(int32_t) * (size_t)n, stream));
    if (bs.masks) QC_TRY(bs.fmask.allocate(ctx, 2 * sizeof(uint32_t) * (size_t)n * bs.T_max, stream));
    QC_TRY(bs.sat.allocate(ctx, sizeof(int32_t) * (size_t)n * bs.T_max, stream));
    QC_TRY(bs.wl.allocate(ctx, 2 * sizeof(int32_t) * (size_t)n * bs.T_max, stream));
    // control block: 8 ints (barrier at [2..3]), then level_new, the per-level work
    // counters (light, heavy) and worklist lengths, each with room for any depth
    // (<= n + 1), then the per-level bit counts (64-bit, at an even offset), then
    // the per-level pulled-item counts of timing mode
    const size_t ctl_ints = 8 + 7 * ((size_t)n + 2);
    QC_TRY(bs.ctl.allocate(ctx, sizeof(int32_t) * ctl_ints, stream));
    return QC_OK;
}

// Queue one launch: the chunk of source words starting at w0, from level `start`
// (2: a fresh chunk), adding into hist (rows rows) and recording its outcome in
// out[0..1] (reset first when reset_out).  stamps: per-level timestamps or null
// (timing mode: the pulled-item counts are then kept in the control block too).
qc_status qc_bfs_launch(qc_graph *g, qc_bfs_scratch &bs, int32_t w0, int32_t start, int32_t *hist, int32_t rows,
                        int32_t *out, bool reset_out, unsigned long long *stamps, cudaStream_t stream) {
    qc_ctx *ctx = g->ctx;
    const int32_t n = g->n;
    const int32_t W = (n + 63) / 64;
    const int32_t wn = (W - w0) < bs.wc ? (W - w0) : bs.wc;
    const int32_t R = (wn + 1) / 2;
    const int32_t T = R >= 32 ? (R + 31) / 32 : 1;
    int G = 32;
    bfs_fn fn = pick(R, bs.masks, &G);
    int per_sm = 0;
    QC_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)fn, 256, 0));
    if (per_sm < 1) {
        qc_set_error(ctx, "BFS kernel cannot be resident on an SM");
        return QC_ERR_CUDA;
    }
    const int items = n * T;
    int blocks = per_sm * qc_coop_sms(ctx);
    if (blocks > qc_ceil_div(items, 8)) blocks = qc_ceil_div(items, 8);
    if (blocks < 1) blocks = 1;
    BfsParams p;
    p.n = n;
    p.row_ptr = g->row_ptr.as<int32_t>();
    p.col_idx = g->col_idx.as<int32_t>();
    p.order = g->order.as<int32_t>();
    p.info = g->oinfo.as<int4>();
    p.comp = g->comp.as<int32_t>();
    p.wcomp = g->wcomp.as<int32_t>();
    p.wmajor = g->wmajor.as<int32_t>();
    p.wmask = g->wmask.as<unsigned long long>();
    p.buf[0] = bs.visB.as<ulonglong2>();
    p.buf[1] = bs.visA.as<ulonglong2>();
    const bool with_masks = bs.masks && G == 32;
    p.fmask[0] = with_masks ? bs.fmask.as<uint32_t>() : nullptr;
    p.fmask[1] = with_masks ? bs.fmask.as<uint32_t>() + (size_t)n * bs.T_max : nullptr;
    p.mask_ratio = bs.mask_ratio;
    p.R = R;
    p.T = T;
    p.w0 = w0;
    p.wn = wn;
    p.W = W;
    p.last_mask = (n % 64) ? (ONES << (n % 64)) : 0ull;
    p.sat = bs.sat.as<int32_t>();
    p.hist = hist;
    p.rows = rows;
    p.first_chunk = (w0 == 0);
    p.start_level = start;
    p.status = out;
    int32_t *c = bs.ctl.as<int32_t>();
    p.bar = reinterpret_cast<unsigned *>(c + 2);
    p.level_new = c + 8;
    p.light_ctr = p.level_new + (n + 2);
    p.heavy_ctr = p.light_ctr + (n + 2);
    p.wl_count = p.heavy_ctr + (n + 2);
    p.level_bits = reinterpret_cast<unsigned long long *>(p.wl_count + (n + 2));
    p.wl[0] = bs.wl.as<int32_t>();
    p.wl[1] = bs.wl.as<int32_t>() + (size_t)n * bs.T_max;
    p.stamp = stamps;
    p.pulled = stamps ? reinterpret_cast<int32_t *>(p.level_bits + (n + 2)) : nullptr;
    p.deg2 = qc_graph_deg2(g);
    p.nnz = g->nnz;
    p.two_hop = bs.two_hop;
    QC_CUDA_TRY(ctx, cudaMemsetAsync(bs.ctl.ptr, 0, bs.ctl.bytes, stream));
    if (reset_out) QC_CUDA_TRY(ctx, cudaMemsetAsync(out, 0, 2 * sizeof(int32_t), stream));
    p.lo = p.row_ptr;
    p.hi = p.row_ptr + 1;
    if (start == 2 && bs.two_hop && 2 * R <= TH_WORDS) {
        // levels 1-2 from the CSR when the graph is sparse enough (decided on the
        // device, by both kernels alike).  With several chunks the set-up reads only
        // the chunk's part of each neighbour list: chunk k's part of N(u) runs from
        // cursor k to cursor k + 1 (cursor 0 = row_ptr), found by binary search from
        // the previous chunk's end; the cursors alternate between two arrays
        if (wn < W && bs.cursor.ptr) {
            const int32_t k = w0 / bs.wc;
            int32_t *cur = bs.cursor.as<int32_t>();
            const int32_t *lo = k == 0 ? p.row_ptr : cur + (size_t)(k & 1) * n;
            int32_t *hi = cur + (size_t)((k + 1) & 1) * n;
            const int64_t bound = std::min<int64_t>(64 * (int64_t)(w0 + wn), n);
            const int cb = std::min(qc_ceil_div(n, 256), 8 * ctx->num_sms);
            chunk_cursor<<<cb, 256, 0, stream>>>(n, p.row_ptr, p.col_idx, lo, (int32_t)bound, hi);
            QC_LAUNCHED(ctx);
            p.lo = lo;
            p.hi = hi;
        }
        const bfs_fn th = with_masks ? bfs_two_hop<true> : bfs_two_hop<false>;
        int th_per_sm = 0;
        QC_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&th_per_sm, (const void *)th, 256, 0));
        int th_blocks = std::max(1, th_per_sm) * qc_coop_sms(ctx);
        if (th_blocks > qc_ceil_div(n, 8)) th_blocks = qc_ceil_div(n, 8);
        th<<<std::max(1, th_blocks), 256, 0, stream>>>(p);
        QC_LAUNCHED(ctx);
    }
    void *args[] = {(void *)&p};
    QC_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void *)fn, dim3(blocks), dim3(256), args, 0, stream));
    QC_LAUNCHED(ctx);
    return QC_OK;
}

// Pulled-item counts of the last timing-mode launch (in the control block).
static const int32_t *pulled_counts(const qc_graph *g, const qc_bfs_scratch &bs) {
    const int32_t n = g->n;
    return bs.ctl.as<int32_t>() + 8 + 4 * (n + 2) + 2 * (n + 2);
}

// The BFS of every source chunk.  sync: each launch is waited for and its outcome
// read (a launch that runs out of histogram rows is relaunched from where it
// stopped; timing mode also records per-launch figures).  Otherwise every launch
// is queued without waiting; the outcome words (g->bfs_out) are read later by
// qc_bfs_settle.
static qc_status bfs_run(qc_graph *g, cudaStream_t stream, bool sync) {
    qc_range range("qc.bfs");
    qc_ctx *ctx = g->ctx;
    const int32_t n = g->n;
    const int32_t W = (n + 63) / 64;
    g->hist_valid = false;
    g->bfs_queued = false;
    g->D = g->nnz > 0 ? 1 : 0;
    QC_TRY(qc_graph_prepare(g, stream));
    QC_TRY(ensure_hist_rows(g, g->nnz > 0 ? 32 : 2, stream));
    if (!g->bfs_out.ptr) QC_TRY(g->bfs_out.allocate(ctx, sizeof(int32_t) * 8, stream));
    if (g->nnz == 0) {
        // no edges: h(0) = 1 for every node, nothing else
        QC_TRY(qc_fill_first_rows(g, stream));
        if (!g->prep_checked) {
            int32_t st = 0;
            QC_CUDA_TRY(ctx, cudaMemcpyAsync(&st, g->prep_ctl.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
            QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
            QC_TRY(qc_graph_prepare_status(g, st));
        }
        g->hist_valid = true;
        return QC_OK;
    }
    qc_bfs_scratch bs;
    QC_TRY(qc_bfs_scratch_init(g, bs, stream));
    int32_t *out = g->bfs_out.as<int32_t>();
    if (!sync) {
        for (int32_t w0 = 0; w0 < W; w0 += bs.wc)
            QC_TRY(qc_bfs_launch(g, bs, w0, 2, g->hist.as<int32_t>(), g->hist_rows, out, w0 == 0, nullptr, stream));
        g->hist_valid = true;
        g->bfs_queued = true;
        return QC_OK;
    }
    qc_pinned pin(ctx);
    QC_TRY(pin.acquire());
    int32_t *h_status = static_cast<int32_t *>(pin.ptr);
    const bool timing = ctx->timing.load();
    qc_event_pair ev;
    qc_buffer stamps;
    if (timing) {
        QC_TRY(ev.create(ctx));
        QC_TRY(stamps.allocate(ctx, sizeof(unsigned long long) * ((size_t)n + 3), stream));
    }
    for (int32_t w0 = 0; w0 < W; w0 += bs.wc) {
        const int32_t wn = (W - w0) < bs.wc ? (W - w0) : bs.wc;
        const int32_t R = (wn + 1) / 2;
        const int32_t T = R >= 32 ? (R + 31) / 32 : 1;
        int32_t start = 2;
        while (true) {
            if (timing) QC_CUDA_TRY(ctx, cudaEventRecord(ev.a, stream));
            QC_TRY(qc_bfs_launch(g, bs, w0, start, g->hist.as<int32_t>(), g->hist_rows, out, true,
                                 timing ? stamps.as<unsigned long long>() : nullptr, stream));
            if (timing) QC_CUDA_TRY(ctx, cudaEventRecord(ev.b, stream));
            QC_CUDA_TRY(ctx, cudaMemcpyAsync(h_status, out, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
            // the preparation's status rides in the same wait (slot 2 of the pinned block)
            if (!g->prep_checked)
                QC_CUDA_TRY(ctx, cudaMemcpyAsync(h_status + 2, g->prep_ctl.ptr, sizeof(int32_t),
                                                 cudaMemcpyDeviceToHost, stream));
            // level stamps and pulled-item counts ride in the same pinned block, after
            // the status words: stamps in its first half, counts in its second
            unsigned long long *h_stamp = reinterpret_cast<unsigned long long *>(
                static_cast<char *>(pin.ptr) + 64);
            const size_t stamp_cap = std::min<size_t>((size_t)n + 3, (QC_PINNED_BYTES / 2 - 64) / 8);
            int32_t *h_pulled = reinterpret_cast<int32_t *>(static_cast<char *>(pin.ptr) + QC_PINNED_BYTES / 2);
            const size_t pulled_cap = std::min<size_t>((size_t)n + 2, (QC_PINNED_BYTES / 2) / 4);
            // the squared-degree sum (bytes 16..23), to repeat the two-hop selection here
            unsigned long long *h_deg2 = reinterpret_cast<unsigned long long *>(static_cast<char *>(pin.ptr) + 16);
            if (timing) {
                QC_CUDA_TRY(ctx, cudaMemcpyAsync(h_deg2, qc_graph_deg2(g), sizeof(unsigned long long),
                                                 cudaMemcpyDeviceToHost, stream));
                QC_CUDA_TRY(ctx, cudaMemcpyAsync(h_stamp, stamps.ptr, sizeof(unsigned long long) * stamp_cap,
                                                 cudaMemcpyDeviceToHost, stream));
                QC_CUDA_TRY(ctx, cudaMemcpyAsync(h_pulled, pulled_counts(g, bs), sizeof(int32_t) * pulled_cap,
                                                 cudaMemcpyDeviceToHost, stream));
            }
            QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
            QC_TRY(qc_debug_take(ctx));
            const int32_t st = h_status[0], reached = h_status[1];
            QC_TRY(qc_graph_prepare_status(g, h_status[2]));
            if (timing) {
                float ms = 0.f;
                QC_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ev.a, ev.b));
                const int passes = reached - start + 1 + (start == 2 ? 1 : 0);
                const double per_pass = qc_bfs_level_model_bytes(n, g->nnz, wn);
                // compulsory HBM bytes: inputs once, histogram rows once, and per level the
                // open rows' segments (read and written) beyond what L2 holds
                double min_bytes = 4.0 * (n + 1) + 4.0 * (double)g->nnz   // CSR
                                   + 4.0 * (n + 1) + 16.0 * n + 4.0 * n    // order, row bounds, components
                                   + 16.0 * W                              // per-word component masks
                                   + 4.0 * n * (reached - start + 1 + (start == 2 && w0 == 0 ? 2 : 0));
                const double tile_segs = T > 1 ? (double)(R - 32 * (T - 1)) : (double)R;   // smallest tile
                for (int l = start; l <= reached && (size_t)l < pulled_cap; ++l) {
                    const double state = 32.0 * tile_segs * (double)h_pulled[l];
                    if (state > (double)ctx->l2_bytes) min_bytes += state - (double)ctx->l2_bytes;
                }
                // a two-hop set-up (the kernels' own rule, evaluated the same way) writes every
                // node's level-2 row once
                const unsigned long long d2 = *h_deg2;
                const bool two_hop =
                    start == 2 && g->hist_rows > 2 && 2 * R <= TH_WORDS &&
                    ((bs.two_hop == 1 && 4ull * d2 <= (unsigned long long)wn * (unsigned long long)g->nnz) ||
                     (bs.two_hop == 2 && d2 < (1ull << 40)));
                if (two_hop) {
                    const double rows2 = 16.0 * (double)R * (double)n;
                    if (rows2 > (double)ctx->l2_bytes) min_bytes += rows2 - (double)ctx->l2_bytes;
                }
                qc_record_kernel(ctx, "bfs_level", ms, passes * per_pass, min_bytes);
                // stamp[l] opens level l (stamp[1] = launch start; the set-up covers levels 1-2);
                // levels past the pinned block's room are left out of the per-level figures
                const unsigned long long *h = h_stamp;
                const int n_stamps = (int)std::min<size_t>((size_t)reached + 2, stamp_cap);
                for (int l = start - 1; l <= reached && l + 1 < n_stamps; ++l) {
                    if (!h[l] || !h[l + 1] || h[l + 1] < h[l]) continue;
                    char name[32];
                    snprintf(name, sizeof name, "bfs_pass_%d", l);
                    qc_record_kernel(ctx, name, (double)(h[l + 1] - h[l]) * 1e-6, per_pass);
                }
            }
            if (st == ST_TIMEOUT) {
                qc_set_error(ctx, "BFS grid barrier timed out (chunk at word %d)", w0);
                return QC_ERR_TIMEOUT;
            }
            if (st == ST_NEED_ROWS) {
                QC_TRY(ensure_hist_rows(g, reached + 1, stream));
                start = reached;
                continue;
            }
            if (reached - 1 > g->D) g->D = reached - 1;
            break;
        }
    }
    g->hist_valid = true;
    return QC_OK;
}

qc_status qc_bfs_histogram(qc_graph *g, cudaStream_t stream) { return bfs_run(g, stream, true); }

qc_status qc_bfs_enqueue(qc_graph *g, cudaStream_t stream) {
    // timing mode reads each launch's figures, so it waits for every launch
    return bfs_run(g, stream, g->ctx->timing.load() || g->nnz == 0);
}

qc_status qc_bfs_settle(qc_graph *g, cudaStream_t stream, bool *redone) {
    *redone = false;
    if (!g->bfs_queued) return QC_OK;
    qc_ctx *ctx = g->ctx;
    qc_pinned pin(ctx);
    QC_TRY(pin.acquire());
    int32_t *h = static_cast<int32_t *>(pin.ptr);
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(h, g->bfs_out.ptr, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    h[2] = 0;
    if (!g->prep_checked)
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(h + 2, g->prep_ctl.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
    g->bfs_queued = false;
    const qc_status dst = qc_debug_take(ctx);
    if (dst != QC_OK) {
        g->hist_valid = false;
        return dst;
    }
    const qc_status pst = qc_graph_prepare_status(g, h[2]);
    if (pst != QC_OK) {
        g->hist_valid = false;
        return pst;
    }
    if (h[0] == ST_TIMEOUT) {
        g->hist_valid = false;
        qc_set_error(ctx, "BFS grid barrier timed out");
        return QC_ERR_TIMEOUT;
    }
    if (h[0] == ST_NEED_ROWS) {
        // a chunk ran out of histogram rows: run the BFS again from fresh rows,
        // waiting for each launch (it grows the rows as it goes)
        *redone = true;
        g->hist.release();
        g->hist_rows = 0;
        return qc_bfs_histogram(g, stream);
    }
    g->D = h[1] - 1;
    return QC_OK;
}

