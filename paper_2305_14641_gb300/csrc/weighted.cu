// Weighted graphs: Section 3.1 makes the distance between adjacent nodes the
// weight of their edge; between any two nodes it is read here as the length of
// the lightest path (for unit weights this is the hop distance).  Lengths are
// real, so the potential of Algorithm 1 is summed pair by pair instead of
// through integer distance bins.
//
// Shortest paths: sources are processed K at a time (K a multiple of 32; by
// default all of them while the block stays within 4 GiB).  dist[v][k] (node-major,
// binary64) holds the best length found from source s0 + k to v.  One
// persistent cooperative launch relaxes, pass after pass,
//     dist[v][k] = min(dist[v][k], min_{u in row v} dist[u][k] + w(v, u))
// (pull over the rows: dist[v][k] is the lightest path from v to the source
// s0 + k along the arcs of row v and onwards; for an undirected graph that is
// also the path from the source to v).  The potential of node v below sums over
// its own row dist[v][.], i.e. over the lengths *from* v, as in the hop path.
// A warp takes a node v and GU groups of 32 sources.  It reads only the
// neighbours whose group changed since the previous pass (chg[u][g] = pass of
// the group's last change), NB such neighbours at a time, so a lane keeps up to
// GU x NB distances in flight and quiet parts of the graph cost one 16-byte load
// per neighbour and pass.  Testing ">= previous pass" rather than "== previous pass" matters: a
// neighbour that changes again in this pass must not hide its earlier change.  Updates are
// in place: a value only ever falls to another path's length, every change is
// seen by the neighbours in the next pass, and a pass without change ends the
// launch (the last change of any (u, group) is read by u's neighbours in the
// pass after it), so the result is the unique fixed point whatever the
// interleaving:
// exactly as Dijkstra's relaxation in the oracle.
//
// Potential: for node v, sum1 = sum_j d^2 e^{-d^2 / 2 sigma^2} and
// sum2 = sum_j e^{...} over the j that v reaches (the self term adds 1 to
// sum2), d = dist[v][j - s0] of each batch, with a table-driven exp (below,
// in integer arithmetic) of d^2 x 1 / (2 sigma^2), sum1 by fused multiply-adds
// and sum2 by binary64 adds.  The sums run over each batch's
// sources in a fixed pattern and over the batches in order, so the result is
// the same on every run; it differs from the oracle's sequential sum over j
// only by rounding (relative 1e-15 or so).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <vector>

#include "qc_device.cuh"
#include "qc_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;
// GU: source groups a warp relaxes together (a multiple of 4); NB: changed
// neighbours a warp reads together.  GU x NB = 16 lengths in flight per lane
// (8 x 2, fewer items of twice the work, measured 2 % slower).
constexpr int GU = 4;
constexpr int NB = 4;
// items a warp takes per counter update (QCGRAPH_SSSP_GRAB overrides): two, measured
// on GB300 for the DC-SBM of N = 16384 with weights, 55.8 ms per weighted step
// against 56.6 with four, 59.6 with one, 60.4 with eight and 66.8 with sixteen
constexpr int GRAB = 2;

struct SsspParams {
    int32_t n;
    const int32_t *col_idx;
    const double *w;
    const int4 *oinfo;             // {node, row start, row end, 0}, heaviest degree bucket first
    double *dist;                  // [n][K]
    int32_t *chg;                  // [n][KGp] pass of the last change of each group (-1: none yet)
    int32_t K, KG, KGp, s0, ns;    // sources s0 .. s0 + ns - 1 (ns <= K); KGp = KG rounded up to GU
    int32_t max_pass;
    int32_t *status;               // [0] state, [1] passes run
    unsigned *bar;
    int32_t *pass_ctr;             // [max_pass + 1] items taken
    int32_t *pass_new;             // [max_pass + 1] some value fell
    int32_t grab;                  // items a warp takes per counter update
};

// The relaxation compares on the integer pipe: non-negative binary64 values
// order like their bit patterns, and a neighbour already at or above the best
// length cannot improve it (w > 0), so most candidates cost an integer compare;
// the rest take one binary64 add.  (An integer-pipe adder, bit-exact, made the
// kernel ALU-bound: 72 against 52 ms for the DC-SBM of N = 16384.)
__device__ __forceinline__ double as_double(unsigned long long b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ unsigned long long bits_of(double x) { return (unsigned long long)__double_as_longlong(x); }

// Most candidates that pass the integer compare still cannot improve: the
// neighbour is closer to the source than v, but not by w.  GB300 runs binary64
// adds at 1/64 of its single-precision rate, and these adds kept its binary64
// pipe two-thirds busy, so a single-precision bound decides first:
// f_down(x) <= x and f_up(x) >= x (the binary64 bits truncated to a float by
// integer operations, clamped to [0, 2^127]), so if the sum of the lower
// bounds of dist[u] and w, rounded down, is above the upper bound of the
// best length, then dist[u] + w > best exactly and its rounded binary64
// value is at least best (rounding is monotone and best is a binary64
// number): no binary64 add is needed.  Only candidates within about 2^-22 of best, or below it, reach
// the binary64 add, whose rounded result alone decides, so the lengths are
// unchanged bit for bit.
__device__ __forceinline__ float f_down(unsigned long long b) {   // b: a non-negative finite binary64
    if (b >= 0x47e0000000000000ull) return 1.7014118346046923e38f;     // 2^127 <= x
    if (b < 0x3810000000000000ull) return 0.0f;                         // x < 2^-126
    return __int_as_float((int)((b >> 29) - (896ull << 23)));           // x truncated to 24 bits
}
// f_down for the candidates, which are below best: where best < 2^127 so are
// they, and the upper clamp is not needed; where best >= 2^127, f_up(best) is
// +inf and the strict test below never skips, whatever this returns.
__device__ __forceinline__ float f_down_below(unsigned long long b) {
    const unsigned hi = (unsigned)(b >> 32);
    const float x = __int_as_float((int)(__funnelshift_l((unsigned)b, hi, 3) - 0xc0000000u));
    return hi < 0x38100000u ? 0.0f : x;
}
__device__ __forceinline__ float f_up(unsigned long long b) {     // b: a non-negative binary64 or +inf
    if (b >= 0x47e0000000000000ull) return __int_as_float(0x7f800000);  // +inf
    if (b < 0x3810000000000000ull) return 1.1754943508222875e-38f;      // 2^-126 > x
    return __int_as_float((int)((b >> 29) - (896ull << 23)) + 1);       // one float step above the truncation
}

// Values that other warps rewrite during a pass are read through L2 only
// (ld.global.cg): L1 is not coherent across SMs, and a line cached there in
// one pass could hand back a length another SM has since lowered.  Reading a
// value that is about to fall is harmless (the change is seen in the next
// pass); the grid barrier makes every write of a pass visible to the next.
__device__ __forceinline__ unsigned long long load_len(const double *dist, size_t i) {
    return (unsigned long long)__ldcg(reinterpret_cast<const long long *>(dist) + i);
}

// One (node, block of GU source groups) item.  The chain of dependent loads is
// kept short: the row bounds come with the node in one 16-byte load, the
// change words of a neighbour's GU groups in one 16-byte load each per 4
// groups, and the item's own lengths only once some neighbour is fresh, issued
// together with the first neighbours' lengths.
__device__ __forceinline__ bool sssp_item(const SsspParams &p, const int pass, const int it, const int lane) {
    constexpr unsigned long long INFB = 0x7ff0000000000000ull;
    const int gb = it / p.n;
    const int4 inf = __ldg(p.oinfo + (it - gb * p.n));
    const int v = inf.x, beg = inf.y, end = inf.z;
    const int g0 = gb * GU;
    unsigned long long mine[GU], best[GU];
    float fbest[GU];                                   // f_up(best)
    bool loaded = false;
    for (int e0 = beg; e0 < end; e0 += 32) {
        const int e = e0 + lane;
        int u = 0;
        float wt = 0.0f;                               // f_down(w)
        int cq[GU];
#pragma unroll
        for (int q = 0; q < GU; ++q) cq[q] = -1;
        if (e < end) {
            u = qcdev::checked_id(__ldg(p.col_idx + e), p.n, qcdev::DBG_WEIGHTED);
            wt = f_down((unsigned long long)__double_as_longlong(__ldg(p.w + e)));
            const int4 *cw = reinterpret_cast<const int4 *>(p.chg + (size_t)u * p.KGp + g0);
#pragma unroll
            for (int q4 = 0; q4 < GU / 4; ++q4) {
                const int4 c = __ldcg(cw + q4);
                cq[4 * q4] = c.x;
                cq[4 * q4 + 1] = c.y;
                cq[4 * q4 + 2] = c.z;
                cq[4 * q4 + 3] = c.w;
            }
        }
        unsigned fm[GU];
        unsigned any_fresh = 0u;
#pragma unroll
        for (int q = 0; q < GU; ++q) {
            fm[q] = __ballot_sync(FULL, cq[q] >= pass - 1);
            any_fresh |= fm[q];
        }
        if (!any_fresh) continue;
        if (!loaded) {
#pragma unroll
            for (int q = 0; q < GU; ++q) {
                mine[q] = (g0 + q < p.KG) ? load_len(p.dist, (size_t)v * p.K + (g0 + q) * 32 + lane) : INFB;
                best[q] = mine[q];
                fbest[q] = f_up(mine[q]);
            }
            loaded = true;
        }
        // up to NB changed neighbours at a time, so that a lane has up to
        // GU x NB lengths in flight
        while (any_fresh) {
            int ub[NB], bb[NB];
            float wb[NB];
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                bb[i] = -1;
                if (any_fresh) {
                    bb[i] = __ffs(any_fresh) - 1;
                    any_fresh &= any_fresh - 1;
                }
                const int src = bb[i] < 0 ? 0 : bb[i];
                ub[i] = __shfl_sync(FULL, u, src);
                wb[i] = __shfl_sync(FULL, wt, src);
            }
            unsigned long long db[NB][GU];
#pragma unroll
            for (int i = 0; i < NB; ++i)
#pragma unroll
                for (int q = 0; q < GU; ++q)
                    db[i][q] = (bb[i] >= 0 && ((fm[q] >> bb[i]) & 1u))
                                   ? load_len(p.dist, (size_t)ub[i] * p.K + (g0 + q) * 32 + lane)
                                   : INFB;
#pragma unroll
            for (int i = 0; i < NB; ++i)
#pragma unroll
                for (int q = 0; q < GU; ++q) {
                    if (db[i][q] >= best[q]) continue;   // w > 0: no shorter path through u
                    if (__fadd_rd(f_down_below(db[i][q]), wb[i]) > fbest[q]) continue;   // dist[u] + w > best
                    const double wv = __ldg(p.w + e0 + bb[i]);
                    const unsigned long long c = bits_of(__dadd_rn(as_double(db[i][q]), wv));
                    if (c < best[q]) {
                        best[q] = c;
                        fbest[q] = f_up(c);
                    }
                }
        }
    }
    if (!loaded) return false;
    bool v_fell = false;
#pragma unroll
    for (int q = 0; q < GU; ++q) {
        if (g0 + q >= p.KG) break;
        const bool fell = best[q] < mine[q];
        if (fell) __stcg(reinterpret_cast<long long *>(p.dist) + (size_t)v * p.K + (g0 + q) * 32 + lane, (long long)best[q]);
        if (__any_sync(FULL, fell)) {
            v_fell = true;
            if (lane == 0) __stcg(p.chg + (size_t)v * p.KGp + g0 + q, pass);
        }
    }
    return v_fell;
}

// Three blocks per SM (80 registers, a few spills) beat two blocks without
// spills (104 registers): 68 against 81-90 ms for the DC-SBM of N = 16384.
__global__ void __launch_bounds__(256, 3) sssp_persistent(const SsspParams p) {
    const int lane = threadIdx.x & 31;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    // pass 0: each source at distance 0 from itself
    for (long long i = tid; i < (long long)p.n * p.K; i += nthreads) {
        const int v = (int)(i / p.K), k = (int)(i - (long long)v * p.K);
        p.dist[i] = (k < p.ns && v == p.s0 + k) ? 0.0 : __longlong_as_double(0x7ff0000000000000ll);
    }
    for (long long i = tid; i < (long long)p.n * p.KGp; i += nthreads) {
        const int v = (int)(i / p.KGp), g = (int)(i - (long long)v * p.KGp);
        const int k = v - p.s0;
        p.chg[i] = (k >= 0 && k < p.ns && (k >> 5) == g) ? 0 : -1;
    }
    if (!qcdev::grid_barrier(p.bar, p.status)) return;
    // An item is (node, block of GU source groups), taken tile-major: every node
    // of one group block (heaviest first, so that no pass ends waiting on a warp
    // that took a hub late) before the next block.  The warps in flight then
    // gather from one block's column of dist (n x GU x 32 x 8 bytes, 16 MiB for
    // n = 16384), which stays in L2 however many sources a launch holds.  A warp
    // takes GRAB consecutive items per counter update and reserves its next
    // GRAB while it works on these.
    const int items = p.n * (p.KGp / GU);
    int pass = 1;
    for (; pass <= p.max_pass; ++pass) {
        bool any = false;
        int base = 0;
        if (lane == 0) base = atomicAdd(p.pass_ctr + pass, p.grab);
        base = __shfl_sync(FULL, base, 0);
        while (base < items) {
            int next = 0;
            if (lane == 0) next = atomicAdd(p.pass_ctr + pass, p.grab);
            for (int j = 0; j < p.grab && base + j < items; ++j)
                any |= sssp_item(p, pass, base + j, lane);
            base = __shfl_sync(FULL, next, 0);
        }
        if (__syncthreads_or(any) && threadIdx.x == 0) p.pass_new[pass] = 1;
        if (!qcdev::grid_barrier(p.bar, p.status)) return;
        if (*(volatile int32_t *)(p.pass_new + pass) == 0) break;
    }
    if (tid == 0) {
        p.status[1] = pass;
        if (pass > p.max_pass) p.status[0] = qcdev::ST_NEED_ROWS;   // not converged within max_pass
    }
}

// exp(-t) for t >= 0 by the table-driven method of Tang (ACM TOMS 15(2), 1989):
// t = a + b/1024 + r with integers a, b (0 <= b < 1024) and 0 <= r < 2^-10, so
// exp(-t) = exp(-a) exp(-b/1024) exp(-r).  On GB300 binary64 arithmetic runs at
// a small fraction of the integer rate, so everything but the last multiply is
// done in 64-bit fixed point:
//   * t (< 708) becomes T = floor(t 2^53), exact to 2^-53 absolute (1 ulp of
//     exp(-t) near 1, less elsewhere); a, b and r are bit fields of T;
//   * exp(-r) = 1 - r (1 - r/2 (1 - r/3 (1 - r/4))) (truncation below 1e-17
//     relative) in Q1.63 by Horner's rule with 64 x 64 -> high 64 products;
//   * times exp(-b/1024), a Q1.63 table built on the host in extended
//     precision;
//   * times exp(-a), a binary64 table: the 53 x 64-bit mantissa product is
//     rounded once to nearest (ties to even) and given exp(-a)'s exponent,
//     all in integer arithmetic.
// About 1 ulp in all.  Above t = 708 the result is subnormal, where the
// binary64 form below (same tables for exp(-a)) is kept; from 745 on it is 0.
// The tables travel as a kernel parameter and each block copies them to shared
// memory: lanes index them at random, which the constant bank would serialise.
struct ExpTables {
    double hi[746];                // exp(-a), a = 0 .. 745
    double lo[64];                 // exp(-b / 64), b = 0 .. 63 (binary64 form)
    unsigned long long fx[1024];   // exp(-b / 1024) in Q1.63, b = 0 .. 1023
    unsigned long long fa[64];     // exp(-a) in Q1.63, a = 0 .. 63 (fixed-point sums)
};

// binary64 form: t = a + b/64 + r, exp(-r) by its Taylor series to degree 6
__device__ __forceinline__ double exp_neg_f64(double t, const ExpTables &T) {
    if (!(t < 745.0)) return 0.0;
    const int k = (int)(t * 64.0);                        // t * 64 is exact; truncation = floor here
    const double r = t - (double)k * (1.0 / 64.0);        // exact (Sterbenz) or r = t when k = 0
    const double y = -r;
    double p = 1.0 / 720.0;
    p = fma(p, y, 1.0 / 120.0);
    p = fma(p, y, 1.0 / 24.0);
    p = fma(p, y, 1.0 / 6.0);
    p = fma(p, y, 0.5);
    p = fma(p, y, 1.0);
    p = fma(p, y, 1.0);
    return T.hi[k >> 6] * T.lo[k & 63] * p;
}

// The block's shared copy of the tables (call before any exp_neg).
__device__ __forceinline__ void load_exp_tables(ExpTables &dst, const ExpTables &src) {
    static_assert(sizeof(ExpTables) % 8 == 0, "tables are 8-byte words");
    const unsigned long long *from = reinterpret_cast<const unsigned long long *>(&src);
    unsigned long long *to = reinterpret_cast<unsigned long long *>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(ExpTables) / 8); i += blockDim.x) to[i] = from[i];
    __syncthreads();
}

// exp(-t) from Tf = floor(t 2^53), t < 708; *fix (if given) receives
// exp(-t) 2^62 rounded down to an integer (within 2 units), 0 from t = 64 on.
__device__ __forceinline__ double exp_neg_fixed(unsigned long long Tf, const ExpTables &T,
                                                unsigned long long *fix = nullptr) {
    constexpr unsigned long long ONE = 1ull << 63;        // 1.0 in Q1.63
    constexpr unsigned long long THIRD = 0x5555555555555555ull;   // floor(2^64 / 3)
    const int a = (int)(Tf >> 53);
    const int b = (int)((Tf >> 43) & 1023);
    const unsigned long long rq = (Tf & ((1ull << 43) - 1)) << 11;   // r 2^64, r < 2^-10
    unsigned long long w = ONE - (rq >> 3);                          // 1 - r/4
    w = ONE - __umul64hi(__umul64hi(rq, THIRD), w);                  // 1 - r/3 (...)
    w = ONE - __umul64hi(rq >> 1, w);                                // 1 - r/2 (...)
    w = ONE - __umul64hi(rq, w);                                     // exp(-r)
    const unsigned long long L = T.fx[b];
    const unsigned long long M = (__umul64hi(L, w) << 1) | ((L * w) >> 63);   // Q1.63, in (0.36, 1]
    if (fix) *fix = a < 64 ? __umul64hi(T.fa[a], M) : 0ull;                  // Q1.63 x Q1.63 -> Q2.62
    // exp(-a) M: the mantissa product (hi:lo, below 2^127) rounded once to 53 bits
    constexpr unsigned long long MANT = (1ull << 52) - 1;
    const unsigned long long hb = (unsigned long long)__double_as_longlong(T.hi[a]);   // normal for a <= 707
    const unsigned long long Ha = ((hb & MANT) | (1ull << 52)) << 11;                 // in [2^63, 2^64)
    const unsigned long long hi = __umul64hi(Ha, M);                                   // in (2^60.5, 2^63)
    const unsigned long long lo = Ha * M;
    const int top = 63 - __clzll((long long)hi);                                       // 60 .. 62
    const int sr = top - 52;
    unsigned long long mant = hi >> sr;
    const unsigned long long rest = hi & ((1ull << sr) - 1), half = 1ull << (sr - 1);
    if (rest > half || (rest == half && (lo != 0 || (mant & 1)))) ++mant;   // to nearest, ties to even
    int eb = (int)(hb >> 52) + top - 62;
    if (mant >> 53) {
        mant >>= 1;
        ++eb;
    }
    return __longlong_as_double((long long)(((unsigned long long)eb << 52) | (mant & MANT)));
}

__device__ __forceinline__ double exp_neg(double t, const ExpTables &T) {
    if (!(t < 708.0)) return exp_neg_f64(t, T);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(t);
    const int e = (int)(bits >> 52);                      // t >= 0: no sign bit
    const unsigned long long m = (bits & ((1ull << 52) - 1)) | (e ? (1ull << 52) : 0ull);
    // Tf = floor(m 2^(e - 1022)) = floor(t 2^53); t < 2^10 keeps it below 2^63
    const int sh = (e ? e : 1) - 1022;
    return exp_neg_fixed(sh >= 0 ? (m << sh) : (sh > -64 ? (m >> -sh) : 0ull), T);
}

// exp(-d2 x inv) for d2 >= 0 and a normal inv > 0 given by its mantissa mi
// (with the leading bit) and ri = 2097 - its exponent field: Tf comes straight
// from the exact 106-bit product of the mantissas, with no binary64 multiply
// (GB300's binary64 pipe is the pair sums' limit).  Products of t >= 2^9, and
// d2 zero or subnormal, take the binary64 route.
__device__ __forceinline__ double exp_neg_product(unsigned long long d2b, unsigned long long mi, int ri,
                                                  double inv, const ExpTables &T) {
    if (d2b == 0) return 1.0;
    const int ed = (int)(d2b >> 52);
    const int r = ri - ed;                                // Tf = (md mi) >> r
    if (ed == 0 || r < 44) return exp_neg(__dmul_rn(__longlong_as_double((long long)d2b), inv), T);
    if (r >= 128) return 1.0;                             // Tf = 0: t < 2^-53
    const unsigned long long md = (d2b & ((1ull << 52) - 1)) | (1ull << 52);
    const unsigned long long hi = __umul64hi(md, mi), lo = md * mi;
    const unsigned long long Tf = r >= 64 ? (hi >> (r - 64)) : ((hi << (64 - r)) | (lo >> r));
    if (Tf >= (708ull << 53)) return exp_neg(__dmul_rn(__longlong_as_double((long long)d2b), inv), T);
    return exp_neg_fixed(Tf, T);
}

// exp_neg_product, and fix = exp(-d2 x inv) 2^62 rounded down as exp_neg_fixed
// gives it: 2^62 where the result is 1, 0 from t = 256 on (the binary64
// route), and for a subnormal d2 (rare) the binary64 result scaled and truncated.
__device__ __forceinline__ double exp_neg_product_fix(unsigned long long d2b, unsigned long long mi, int ri,
                                                      double inv, const ExpTables &T, unsigned long long &fix) {
    constexpr unsigned long long ONE62 = 1ull << 62;
    fix = ONE62;
    if (d2b == 0) return 1.0;
    const int ed = (int)(d2b >> 52);
    const int r = ri - ed;
    if (ed == 0) {
        const double e = exp_neg(__dmul_rn(__longlong_as_double((long long)d2b), inv), T);
        fix = (unsigned long long)(e * 4611686018427387904.0);   // e 2^62 (exact), truncated
        return e;
    }
    fix = 0ull;
    if (r < 44) return exp_neg(__dmul_rn(__longlong_as_double((long long)d2b), inv), T);
    fix = ONE62;
    if (r >= 128) return 1.0;
    const unsigned long long md = (d2b & ((1ull << 52) - 1)) | (1ull << 52);
    const unsigned long long hi = __umul64hi(md, mi), lo = md * mi;
    const unsigned long long Tf = r >= 64 ? (hi >> (r - 64)) : ((hi << (64 - r)) | (lo >> r));
    if (Tf >= (708ull << 53)) {
        fix = 0ull;
        return exp_neg(__dmul_rn(__longlong_as_double((long long)d2b), inv), T);
    }
    return exp_neg_fixed(Tf, T, &fix);
}

// acc[s][v] += (sum1, sum2) over the batch's sources for node v: a warp per node,
// lane l takes sources l, l + 32, ... in order (each distance read once for up
// to SGRP sigma values), then a butterfly over the lanes (every lane ends with
// the same total) and one add into the running sums, so the result is the same
// on every run.
constexpr int SGRP = 8;
// Three blocks per SM (80 registers) by a hair over two (92 registers).
__global__ void __launch_bounds__(256, 3) wpot_accumulate(int32_t n, int32_t K, int32_t ns, const double *dist, int32_t S,
                                const double *den, double2 *acc, const __grid_constant__ ExpTables Tp) {
    __shared__ ExpTables T;
    load_exp_tables(T, Tp);
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int v = warp; v < n; v += nwarps) {
        const double *row = dist + (size_t)v * K;
        for (int s0 = 0; s0 < S; s0 += SGRP) {
            double inv[SGRP], s1[SGRP], s2[SGRP];
            unsigned long long im[SGRP];
            int ir[SGRP];
#pragma unroll
            for (int j = 0; j < SGRP; ++j) {
                inv[j] = (s0 + j < S) ? 1.0 / den[s0 + j] : 1.0;   // one division per node and sigma
                const unsigned long long ib = (unsigned long long)__double_as_longlong(inv[j]);
                im[j] = (ib & ((1ull << 52) - 1)) | (1ull << 52);
                ir[j] = 2097 - (int)(ib >> 52);
                s1[j] = 0.0;
                s2[j] = 0.0;
            }
            for (int k = lane; k < ns; k += 32) {
                const double d = row[k];
                if (__double_as_longlong(d) >= 0x7ff0000000000000ll) continue;   // unreachable (+inf)
                const double d2 = __dmul_rn(d, d);
                const unsigned long long d2b = (unsigned long long)__double_as_longlong(d2);
#pragma unroll
                for (int j = 0; j < SGRP; ++j) {
                    if (s0 + j < S) {
                        const double e = exp_neg_product(d2b, im[j], ir[j], inv[j], T);
                        s1[j] = fma(d2, e, s1[j]);
                        s2[j] = __dadd_rn(s2[j], e);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < SGRP; ++j) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    s1[j] = __dadd_rn(s1[j], __shfl_xor_sync(FULL, s1[j], off));
                    s2[j] = __dadd_rn(s2[j], __shfl_xor_sync(FULL, s2[j], off));
                }
                if (lane == 0 && s0 + j < S) {
                    double2 a = acc[(size_t)(s0 + j) * n + v];
                    a.x = __dadd_rn(a.x, s1[j]);
                    a.y = __dadd_rn(a.y, s2[j]);
                    acc[(size_t)(s0 + j) * n + v] = a;
                }
            }
        }
    }
}

// (hi:lo) += b, 128-bit unsigned
__device__ __forceinline__ void add128(unsigned long long &lo, unsigned long long &hi, unsigned long long b) {
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(lo), "+l"(hi) : "l"(b));
}
// (hi 2^64 + lo) 2^-q as binary64: the product is exact, the sum rounds once
__device__ __forceinline__ double fixed_to_double(unsigned long long lo, unsigned long long hi, double scale) {
    return __dmul_rn(__fma_rn(__ull2double_rn(hi), 18446744073709551616.0, __ull2double_rn(lo)), scale);
}

// Symmetric pair sums, for undirected graphs whose sources a launch holds all
// at once: the length from v to j and the one from j to v are the same
// shortest-path length (accumulated from opposite ends, so they may differ in
// the last bits), and each unordered pair's exponential is evaluated once for
// both nodes' sums.  Work: strips of 32 rows (4 per warp) against segments of
// SYM_SEG columns at or right of the strip's first node, lanes across the
// columns.  A pair (v, j) with v in the strip adds to v's row sums; when j lies
// right of the strip it also adds to j's column sums.  Node v's sums are then
// its strip's row sums (columns from the strip's first node on) plus the
// column sums of the strips left of it, which covers every j once.
//   rows: butterfly over the lanes of d^2 e (binary64) and of e 2^57 (integer),
//         added into per-row shared accumulators, written per (item, row);
//   columns: per lane over the warp's 4 rows, a fused multiply-add for sum1 and
//         e 2^61 in integers for sum2, then the 8 warps in order through shared
//         memory, written per (strip, column).
// sum2 in integers is exact but for the truncation of each term (2^-57 or
// 2^-61); with sum2 >= 1 (the self term) that is within n 2^-57 relative.  The
// partial sums are reduced in a fixed order (wpot_sym_reduce), so the result is
// the same on every run.  GB300's binary64 pipe does about one operation per
// ordered pair and sigma instead of two, and the exponential half as often.
constexpr int SYM_ROWS = 32;
constexpr int SYM_SEG = 1024;
constexpr int SYM_SG = 2;          // sigmas per launch

__global__ void __launch_bounds__(256, 3) wpot_sym(int32_t n, int32_t K, const double *dist, int32_t S,
                                                   const double *den, int32_t nsegm, int32_t items,
                                                   int32_t *item_ctr, double2 *prow, double2 *pcol,
                                                   const __grid_constant__ ExpTables Tp) {
    constexpr int RW = SYM_ROWS / 8;   // rows per warp
    __shared__ ExpTables T;
    __shared__ double cs1w[8][32][SYM_SG];
    __shared__ unsigned long long cs2w[8][32][SYM_SG];
    __shared__ int s_item;
    __shared__ double s_inv[SYM_SG];                 // 1 / (2 sigma^2), for the rare binary64 route
    if (threadIdx.x < SYM_SG) s_inv[threadIdx.x] = ((int)threadIdx.x < S) ? 1.0 / den[threadIdx.x] : 1.0;
    load_exp_tables(T, Tp);                          // (its barrier publishes s_inv too)
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned long long im[SYM_SG];
    int ir[SYM_SG];
#pragma unroll
    for (int s = 0; s < SYM_SG; ++s) {
        const unsigned long long ib = (unsigned long long)__double_as_longlong(s_inv[s]);
        im[s] = (ib & ((1ull << 52) - 1)) | (1ull << 52);
        ir[s] = 2097 - (int)(ib >> 52);
    }
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(item_ctr, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= items) break;
        const int strip = it / nsegm, c = it - strip * nsegm;
        const int i0 = strip * SYM_ROWS;
        const int jb = i0 + c * SYM_SEG;
        if (jb >= n) continue;
        const int je = min(n, jb + SYM_SEG);
        // this lane's part of the warp's rows over the item's columns: sum1 by
        // fused multiply-adds, sum2 as e 2^57 in integers (at most 32 chunks of
        // one term each: below 2^62)
        double rs1[RW][SYM_SG];
        unsigned long long rs2[RW][SYM_SG];
#pragma unroll
        for (int rr = 0; rr < RW; ++rr)
#pragma unroll
            for (int s = 0; s < SYM_SG; ++s) {
                rs1[rr][s] = 0.0;
                rs2[rr][s] = 0ull;
            }
        for (int j0 = jb; j0 < je; j0 += 32) {
            const bool diag = j0 == i0;                  // the strip's own columns: rows only
            const int j = j0 + lane;
            const bool jok = j < je;
            double cs1[SYM_SG];
            unsigned long long cs2[SYM_SG];
#pragma unroll
            for (int s = 0; s < SYM_SG; ++s) {
                cs1[s] = 0.0;
                cs2[s] = 0ull;
            }
#pragma unroll
            for (int rr = 0; rr < RW; ++rr) {
                const int v = i0 + warp * RW + rr;
                const double d = (v < n && jok) ? dist[(size_t)v * K + j] : __longlong_as_double(0x7ff0000000000000ll);
                // unreachable (+inf), or outside the item; an integer compare keeps
                // it off the binary64 pipe
                if (__double_as_longlong(d) >= 0x7ff0000000000000ll) continue;
                const double d2 = __dmul_rn(d, d);
                const unsigned long long d2b = (unsigned long long)__double_as_longlong(d2);
#pragma unroll
                for (int s = 0; s < SYM_SG; ++s) {
                    if (s >= S) continue;
                    unsigned long long fx;
                    const double e = exp_neg_product_fix(d2b, im[s], ir[s], s_inv[s], T, fx);
                    rs1[rr][s] = fma(d2, e, rs1[rr][s]);
                    rs2[rr][s] += fx >> 5;
                    if (!diag) {
                        cs1[s] = fma(d2, e, cs1[s]);
                        cs2[s] += fx >> 1;                   // the warp's rows: at most 2^63
                    }
                }
            }
            if (!diag) {
#pragma unroll
                for (int s = 0; s < SYM_SG; ++s) {
                    cs1w[warp][lane][s] = cs1[s];
                    cs2w[warp][lane][s] = cs2[s];
                }
                __syncthreads();
                for (int i = threadIdx.x; i < 32 * SYM_SG; i += blockDim.x) {
                    const int l = i / SYM_SG, s = i - l * SYM_SG;
                    double a = cs1w[0][l][s];
                    unsigned long long lo = cs2w[0][l][s], hi = 0ull;
                    for (int w = 1; w < 8; ++w) {
                        a = __dadd_rn(a, cs1w[w][l][s]);
                        add128(lo, hi, cs2w[w][l][s]);
                    }
                    if (j0 + l < je)
                        pcol[((size_t)strip * n + j0 + l) * SYM_SG + s] = make_double2(a, fixed_to_double(lo, hi, 0x1p-61));
                }
                __syncthreads();
            }
        }
        // the rows' totals over the lanes (every lane ends with the same sums)
#pragma unroll
        for (int rr = 0; rr < RW; ++rr)
#pragma unroll
            for (int s = 0; s < SYM_SG; ++s) {
                double x = rs1[rr][s];
                unsigned long long lo = rs2[rr][s], hi = 0ull;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    x = __dadd_rn(x, __shfl_xor_sync(FULL, x, off));
                    const unsigned long long olo = __shfl_xor_sync(FULL, lo, off), ohi = __shfl_xor_sync(FULL, hi, off);
                    add128(lo, hi, olo);
                    hi += ohi;
                }
                if (lane == 0)
                    prow[((size_t)it * SYM_ROWS + warp * RW + rr) * SYM_SG + s] =
                        make_double2(x, fixed_to_double(lo, hi, 0x1p-57));
            }
    }
}

// acc[s][v] = node v's row sums over its strip's segments, then the column
// sums of every strip left of it, in that order.
__global__ void wpot_sym_reduce(int32_t n, int32_t S, int32_t nsegm, const double2 *prow, const double2 *pcol,
                                double2 *acc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n * SYM_SG; i += gridDim.x * blockDim.x) {
        const int v = i / SYM_SG, s = i - v * SYM_SG;
        if (s >= S) continue;
        const int strip = v / SYM_ROWS, r = v - strip * SYM_ROWS;
        double a1 = 0.0, a2 = 0.0;
        for (int c = 0; c < nsegm && strip * SYM_ROWS + c * SYM_SEG < n; ++c) {
            const double2 x = prow[((size_t)(strip * nsegm + c) * SYM_ROWS + r) * SYM_SG + s];
            a1 = __dadd_rn(a1, x.x);
            a2 = __dadd_rn(a2, x.y);
        }
        for (int I = 0; I < strip; ++I) {
            const double2 x = pcol[((size_t)I * n + v) * SYM_SG + s];
            a1 = __dadd_rn(a1, x.x);
            a2 = __dadd_rn(a2, x.y);
        }
        acc[(size_t)s * n + v] = make_double2(a1, a2);
    }
}

__global__ void wpot_final(int32_t n, int32_t S, const double *den, const double2 *acc, double *V) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S * n; i += gridDim.x * blockDim.x) {
        const int s = i / n;
        const double2 a = acc[i];
        V[i] = __ddiv_rn(__ddiv_rn(a.x, a.y), den[s]);
    }
}

enum : int32_t { BAD_WEIGHT = 1, BAD_MIRROR = 2 };

// Positive finite weights; for an undirected graph w(v, u) = w(u, v).
__global__ void check_weights(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const double *w,
                              bool symmetric, int32_t *err) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int bad = 0;
    for (int v = warp; v < n; v += nwarps) {
        for (int e = row_ptr[v] + lane; e < row_ptr[v + 1]; e += 32) {
            const double x = w[e];
            if (!(x > 0.0) || !(x < 1e308)) bad |= BAD_WEIGHT;
            if (!symmetric) continue;
            const int u = qcdev::checked_id(col_idx[e], n, qcdev::DBG_WEIGHTED);
            int lo = row_ptr[u], hi = row_ptr[u + 1] - 1;
            bool same = false;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const int y = col_idx[mid];
                if (y == v) { same = (w[mid] == x); break; }
                if (y < v) lo = mid + 1; else hi = mid - 1;
            }
            if (!same) bad |= BAD_MIRROR;
        }
    }
    bad = __reduce_or_sync(FULL, bad);
    if (lane == 0 && bad) atomicOr(err, bad);
}

// Sources per shortest-path launch.  Each pass of a launch ends at a grid
// barrier whose cost does not grow with K, and the tile-major item order keeps
// the gathers in L2 whatever K is, so a launch takes every source while the
// distance block stays within 4 GiB (n <= 23170), else an even split of them
// into blocks below that.  QCGRAPH_SSSP_SOURCES overrides it.
// The exponential's tables, from the C library's exp in extended precision
// (long double), each rounded once.
void fill_exp_tables(ExpTables &T) {
    for (int a = 0; a < 746; ++a) T.hi[a] = (double)std::exp(-(long double)a);
    for (int b = 0; b < 64; ++b) T.lo[b] = (double)std::exp(-(long double)b / 64.0L);
    for (int b = 0; b < 1024; ++b)   // <= 2^63, rounded to the nearest integer
        T.fx[b] = (unsigned long long)(std::ldexp(std::exp(-(long double)b / 1024.0L), 63) + 0.5L);
    for (int a = 0; a < 64; ++a)     // <= 2^63, rounded to the nearest integer
        T.fa[a] = (unsigned long long)(std::ldexp(std::exp(-(long double)a), 63) + 0.5L);
}

__global__ void exp_neg_kernel(int64_t n, const double *t, double *out, const __grid_constant__ ExpTables Tp) {
    __shared__ ExpTables T;
    load_exp_tables(T, Tp);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = exp_neg(t[i], T);
}

int32_t sources_per_batch(int32_t n) {
    const int64_t cover = ((int64_t)n + 31) / 32 * 32;
    int64_t K;
    if (const char *env = getenv("QCGRAPH_SSSP_SOURCES")) {
        K = atoll(env) / 32 * 32;
    } else {
        const int64_t target = std::max<int64_t>((int64_t)(((size_t)4 << 30) / (8 * (size_t)std::max(n, 1))), 32);
        const int64_t batches = (cover + target - 1) / target;
        K = ((cover + batches - 1) / batches + 31) / 32 * 32;
    }
    if (K < 32) K = 32;
    // the items of a pass, n x ceil(K / 128), stay below 2^30
    const int64_t k_items = std::max<int64_t>((((int64_t)1 << 30) / std::max(n, 1)) / GU * 32 * GU, 32);
    return (int32_t)std::min<int64_t>(std::min<int64_t>(K, k_items), cover);
}

// The symmetric pair sums (wpot_sym) of a distance block that holds every
// source, SYM_SG sigmas per launch, into acc[s][v].
qc_status wpot_symmetric(qc_ctx *ctx, int32_t n, int32_t K, const double *dist, int32_t n_sigma, const double *dden,
                         double2 *acc, const ExpTables &etab, cudaStream_t stream) {
    const int32_t strips = qc_ceil_div(n, SYM_ROWS);
    const int32_t nsegm = qc_ceil_div(n, SYM_SEG);
    const int32_t items = strips * nsegm;
    const int32_t groups = qc_ceil_div(n_sigma, SYM_SG);
    qc_buffer prow, pcol, ctr;
    QC_TRY(prow.allocate(ctx, sizeof(double2) * (size_t)items * SYM_ROWS * SYM_SG, stream));
    QC_TRY(pcol.allocate(ctx, sizeof(double2) * (size_t)strips * n * SYM_SG, stream));
    QC_TRY(ctr.allocate(ctx, sizeof(int32_t) * (size_t)groups, stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(ctr.ptr, 0, ctr.bytes, stream));
    int per_sm = 0;
    QC_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)wpot_sym, 256, 0));
    const int blocks = std::max(1, std::min(std::max(per_sm, 1) * ctx->num_sms, items));
    const int rb = std::max(1, std::min(qc_ceil_div((int64_t)n * SYM_SG, 256), 4 * ctx->num_sms));
    for (int32_t gi = 0; gi < groups; ++gi) {
        const int32_t s0 = gi * SYM_SG;
        const int32_t S = std::min(SYM_SG, n_sigma - s0);
        wpot_sym<<<blocks, 256, 0, stream>>>(n, K, dist, S, dden + s0, nsegm, items, ctr.as<int32_t>() + gi,
                                             prow.as<double2>(), pcol.as<double2>(), etab);
        QC_LAUNCHED(ctx);
        wpot_sym_reduce<<<rb, 256, 0, stream>>>(n, S, nsegm, prow.as<double2>(), pcol.as<double2>(),
                                                acc + (size_t)s0 * n);
        QC_LAUNCHED(ctx);
    }
    return QC_OK;
}

}  // namespace

extern "C" qc_status qc_graph_set_weights(qc_graph *g, const double *w, uint32_t flags, void *stream_) {
    if (!g || (!w && g->nnz > 0)) return QC_ERR_INVALID_ARG;
    qc_ctx *ctx = g->ctx;
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    qc_buffer nb;
    const size_t bytes = sizeof(double) * (size_t)(g->nnz > 0 ? g->nnz : 1);
    QC_TRY(nb.allocate(ctx, bytes, stream));
    if (g->nnz > 0)
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(nb.ptr, w, sizeof(double) * (size_t)g->nnz,
                                         (flags & QC_PTR_DEVICE) ? cudaMemcpyDeviceToDevice
                                                                 : cudaMemcpyHostToDevice,
                                         stream));
    if ((flags & QC_VALIDATE) && g->nnz > 0) {
        qc_buffer err;
        QC_TRY(err.allocate(ctx, sizeof(int32_t), stream));
        QC_CUDA_TRY(ctx, cudaMemsetAsync(err.ptr, 0, sizeof(int32_t), stream));
        const int blocks = qc_ceil_div(g->n, 8) < 8 * ctx->num_sms ? qc_ceil_div(g->n, 8) : 8 * ctx->num_sms;
        check_weights<<<blocks, 256, 0, stream>>>(g->n, g->row_ptr.as<int32_t>(), g->col_idx.as<int32_t>(),
                                                  nb.as<double>(), !g->directed, err.as<int32_t>());
        QC_LAUNCHED(ctx);
        qc_pinned pin(ctx);
        QC_TRY(pin.acquire());
        int32_t *h = static_cast<int32_t *>(pin.ptr);
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(h, err.ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
        QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
        QC_TRY(qc_debug_take(ctx));
        if (h[0]) {
            qc_set_error(ctx, "invalid weights (flags 0x%x):%s%s", h[0],
                         (h[0] & BAD_WEIGHT) ? " not finite and > 0;" : "",
                         (h[0] & BAD_MIRROR) ? " w(u, v) != w(v, u) in an undirected graph;" : "");
            return QC_ERR_INVALID_GRAPH;
        }
    }
    QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));   // a host source may be freed on return
    g->weights = std::move(nb);
    g->weighted = true;
    return QC_OK;
}

extern "C" qc_status qc_potential_weighted(qc_graph *g, const double *sigmas, int32_t n_sigma, double *V_out,
                                           void *stream_) {
    qc_range range("qc.potential_weighted");
    if (!g || !sigmas || n_sigma < 1 || !V_out) return QC_ERR_INVALID_ARG;
    qc_ctx *ctx = g->ctx;
    if (!g->weighted) {
        qc_set_error(ctx, "qc_potential_weighted: the graph has no weights (qc_graph_set_weights)");
        return QC_ERR_INVALID_ARG;
    }
    for (int32_t s = 0; s < n_sigma; ++s)
        if (!qc_sigma_ok(sigmas[s])) {
            qc_set_error(ctx, "qc_potential_weighted: sigma[%d] = %g is not finite and > 0", s, sigmas[s]);
            return QC_ERR_INVALID_ARG;
        }
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const int32_t n = g->n;
    const int32_t K = sources_per_batch(n);
    const int32_t KG = K / 32;
    const void *kern = (const void *)sssp_persistent;
    const int32_t KGp = (KG + GU - 1) / GU * GU;
    QC_TRY(qc_graph_prepare(g, stream));     // the degree order of the nodes
    const int32_t max_pass = n + 1;     // a lightest path has at most n - 1 arcs
    std::vector<double> den(n_sigma);
    for (int32_t s = 0; s < n_sigma; ++s) den[s] = 2.0 * (sigmas[s] * sigmas[s]);
    ExpTables etab;
    fill_exp_tables(etab);
    qc_buffer dist, chg, ctl, acc, dden;
    QC_TRY(dist.allocate(ctx, sizeof(double) * (size_t)n * K, stream));
    QC_TRY(chg.allocate(ctx, sizeof(int32_t) * (size_t)n * KGp, stream));
    QC_TRY(ctl.allocate(ctx, sizeof(int32_t) * (8 + 2 * ((size_t)max_pass + 1)), stream));
    QC_TRY(acc.allocate(ctx, sizeof(double2) * (size_t)n_sigma * n, stream));
    QC_CUDA_TRY(ctx, cudaMemsetAsync(acc.ptr, 0, acc.bytes, stream));
    QC_TRY(dden.allocate(ctx, sizeof(double) * n_sigma, stream));
    QC_CUDA_TRY(ctx, cudaMemcpyAsync(dden.ptr, den.data(), sizeof(double) * n_sigma, cudaMemcpyHostToDevice,
                                     stream));
    int per_sm = 0;
    QC_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0));
    if (per_sm < 1) {
        qc_set_error(ctx, "shortest-path kernel cannot be resident on an SM");
        return QC_ERR_CUDA;
    }
    int blocks = per_sm * qc_coop_sms(ctx);
    const int want = qc_ceil_div((int64_t)n * (KGp / GU), 8);
    if (blocks > want) blocks = want;
    if (blocks < 1) blocks = 1;
    qc_pinned pin(ctx);
    QC_TRY(pin.acquire());
    int32_t *h = static_cast<int32_t *>(pin.ptr);
    const int pblocks = std::max(1, std::min(qc_ceil_div(n, 8), 8 * ctx->num_sms));
    // an undirected graph whose sources all fit one block takes the symmetric
    // pair sums (QCGRAPH_WPOT_SYM=0 keeps the per-node form)
    const char *sym_env = getenv("QCGRAPH_WPOT_SYM");
    const bool sym = !g->directed && K >= n && !(sym_env && sym_env[0] == '0');
    for (int32_t s0 = 0; s0 < n; s0 += K) {
        SsspParams p;
        p.n = n;
        p.col_idx = g->col_idx.as<int32_t>();
        p.w = g->weights.as<double>();
        p.oinfo = g->oinfo.as<int4>();
        p.dist = dist.as<double>();
        p.chg = chg.as<int32_t>();
        p.K = K;
        p.KG = KG;
        p.KGp = KGp;
        p.s0 = s0;
        p.ns = std::min(K, n - s0);
        p.max_pass = max_pass;
        p.status = ctl.as<int32_t>();
        p.bar = reinterpret_cast<unsigned *>(ctl.as<int32_t>() + 2);
        p.pass_ctr = ctl.as<int32_t>() + 8;
        p.pass_new = p.pass_ctr + (max_pass + 1);
        p.grab = GRAB;
        if (const char *env = getenv("QCGRAPH_SSSP_GRAB")) p.grab = std::max(1, std::min(64, atoi(env)));
        QC_CUDA_TRY(ctx, cudaMemsetAsync(ctl.ptr, 0, ctl.bytes, stream));
        void *args[] = {(void *)&p};
        QC_CUDA_TRY(ctx, cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(256), args,
                                                     0, stream));
        QC_LAUNCHED(ctx);
        QC_CUDA_TRY(ctx, cudaMemcpyAsync(h, ctl.ptr, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
        QC_CUDA_TRY(ctx, cudaStreamSynchronize(stream));
        QC_TRY(qc_debug_take(ctx));
        if (h[0] == qcdev::ST_TIMEOUT) {
            qc_set_error(ctx, "shortest paths: grid barrier timed out (sources from %d)", s0);
            return QC_ERR_TIMEOUT;
        }
        if (h[0] != qcdev::ST_DONE) {
            qc_set_error(ctx, "shortest paths did not settle within %d passes", max_pass);
            return QC_ERR_CUDA;
        }
        if (sym) {
            QC_TRY(wpot_symmetric(ctx, n, K, dist.as<double>(), n_sigma, dden.as<double>(), acc.as<double2>(), etab,
                                  stream));
        } else {
            wpot_accumulate<<<pblocks, 256, 0, stream>>>(n, K, p.ns, dist.as<double>(), n_sigma,
                                                         dden.as<double>(), acc.as<double2>(), etab);
            QC_LAUNCHED(ctx);
        }
    }
    const int fb = std::max(1, std::min(qc_ceil_div((int64_t)n_sigma * n, 256), 2 * ctx->num_sms));
    wpot_final<<<fb, 256, 0, stream>>>(n, n_sigma, dden.as<double>(), acc.as<double2>(), V_out);
    QC_LAUNCHED(ctx);
    return QC_OK;
}

extern "C" qc_status qc_selftest_arith(qc_ctx *ctx, int32_t op, const double *x, const double *y, double *out,
                                       int64_t n, void *stream_) {
    (void)y;
    if (!ctx || n < 0 || op != QC_ARITH_EXP_NEG) return QC_ERR_INVALID_ARG;
    if (n > 0 && (!x || !out)) return QC_ERR_INVALID_ARG;
    if (n == 0) return QC_OK;
    cudaStream_t stream = qc_stream(stream_);
    QC_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4 * (int64_t)ctx->num_sms);
    ExpTables etab;
    fill_exp_tables(etab);
    exp_neg_kernel<<<blocks, 256, 0, stream>>>(n, x, out, etab);
    QC_LAUNCHED(ctx);
    return QC_OK;
}
