// polar_kernels.cu -- list-CRC decoding of polar codes over the unrolled
// Fast-SSC tree, for GB300 (sm_103a).
//
// One frame is decoded by a group of W warps (W = 1, 2, 4); a CTA of up to
// 512 threads holds several groups and every group loops over frames
// (persistent). The groups of a CTA run the same schedule, and while all of
// them hold a frame a CTA barrier before every register subtree keeps them on
// the same instructions (they share instruction fetches). All L paths of a frame
// advance through the schedule in lockstep, so:
//
//  * alpha stage j (kSubLog <= j < n) holds one row of 2^j LLRs per physical
//    slot. F and G (Eq. (1), (2)) read stage j+1 through the path's index-
//    table entry and always write the path's own row of stage j: at that
//    moment stage j is dead for every path. A fork only copies the parent's
//    16-byte index row -- the lazy copy of Sec. IV-A -- never LLRs.
//  * beta is bit-packed. Left-child outputs (BL[j]) sit behind a second
//    index table (Sec. IV-B); the right-child / root output (BR) is consumed
//    by the Combine (Eq. (3)) that follows at once and needs none.
//  * every subtree of at most 16 bits is one operation (OP_SUB) run by warp 0
//    with one lane per path: its LLRs, betas and penalty stay in registers, a
//    fork moves a path's state from its parent lane by warp shuffles, and only
//    the subtree root touches memory. An inner node of 32 bits whose children
//    are such subtrees is one operation too (F and G from its input row, both
//    subtrees, Combine). Leaves of more than 16 bits also run one lane per
//    path (vectorised scans of the path's row).
//  * a forking leaf (Sec. III-C..E) produces keys (penalty, source * C +
//    candidate) in the source lane. The L smallest survive (Algorithm 1). With
//    a full list the L-th key is at most the largest source-best key, so only
//    the later candidates below it are sorted and merged with the sorted best
//    column; otherwise columns are merged in while their minimum is below the
//    current L-th key. Survivors are numbered in (source, candidate) order by
//    a warp prefix scan.
//  * buffers that do not fit the shared-memory budget live in a per-group
//    global scratch region (L2-resident in practice).
//  * the final pick (Sec. II-B) checks each path's CRC with byte tables of
//    the syndrome of every codeword bit, and writes the winner's payload.
//
// Float sums of many terms (Rate-0, repetition) use the pairwise tree
// s[i] = x[i] + x[i + n/2]; sums of least-reliable-bit terms run left to
// right in rank order; every new penalty is parent + increment. int8 LLRs
// use saturated G and exact integer penalties.

#include <algorithm>
#include <type_traits>

#include "polar_internal.h"

namespace polar {
namespace {

constexpr uint32_t FULL = 0xffffffffu;

template <typename T> struct Arith;

template <> struct Arith<float> {
    typedef float P;
    typedef unsigned long long K;                 // key: penalty bits << 32 | candidate index
    static constexpr K KINF = ~0ull;
    static __device__ __forceinline__ K mk(float p, uint32_t idx) { return ((K)__float_as_uint(p) << 32) | idx; }
    static __device__ __forceinline__ float kpen(K k) { return __uint_as_float((uint32_t)(k >> 32)); }
    static __device__ __forceinline__ uint32_t kidx(K k) { return (uint32_t)k; }
    static __device__ __forceinline__ uint32_t pbits(float p) { return __float_as_uint(p); }
    static __device__ __forceinline__ float to_out(float p) { return p; }
    static __device__ __forceinline__ uint32_t absbits(float a) { return __float_as_uint(fabsf(a)); }
    static __device__ __forceinline__ float unabs(uint32_t b) { return __uint_as_float(b); }
    static __device__ __forceinline__ float negpart(float a) { return a < 0.f ? -a : 0.f; }
    static __device__ __forceinline__ float pospart(float a) { return a > 0.f ? a : 0.f; }
    static __device__ __forceinline__ float val(float a) { return a; }
};

template <> struct Arith<int8_t> {
    typedef int P;
    typedef uint32_t K;                           // penalty < 2^20 << 8 | candidate index < 256
    static constexpr K KINF = ~0u;
    static __device__ __forceinline__ K mk(int p, uint32_t idx) { return ((uint32_t)p << 8) | idx; }
    static __device__ __forceinline__ int kpen(K k) { return (int)(k >> 8); }
    static __device__ __forceinline__ uint32_t kidx(K k) { return k & 0xFFu; }
    static __device__ __forceinline__ uint32_t pbits(int p) { return (uint32_t)p; }
    static __device__ __forceinline__ float to_out(int p) { return (float)p; }
    static __device__ __forceinline__ uint32_t absbits(int a) { return (uint32_t)(a < 0 ? -a : a); }
    static __device__ __forceinline__ int unabs(uint32_t b) { return (int)b; }
    static __device__ __forceinline__ int negpart(int a) { return a < 0 ? -a : 0; }
    static __device__ __forceinline__ int pospart(int a) { return a > 0 ? a : 0; }
    static __device__ __forceinline__ int val(int8_t a) { return (int)a; }
};

// ---- F and G (Eq. (1), (2)) ------------------------------------------------
// float: F = sign(a) sign(b) min(|a|, |b|); the sign is taken from the sign
// bits, which can only differ from a comparison when the result is zero.
__device__ __forceinline__ float f_op(float a, float b) {
    float m = fminf(fabsf(a), fabsf(b));
    return __uint_as_float(__float_as_uint(m) | ((__float_as_uint(a) ^ __float_as_uint(b)) & 0x80000000u));
}
__device__ __forceinline__ float g_op(float a, float b, uint32_t beta) {
    return b + __uint_as_float(__float_as_uint(a) ^ (beta << 31));
}
// Four int8 lanes in one word: F = max(min(a,b), -max(a,b)).
__device__ __forceinline__ uint32_t f4(uint32_t a, uint32_t b) {
    return __vmaxs4(__vmins4(a, b), __vneg4(__vmaxs4(a, b)));
}
// G on four int8 lanes; nib holds the four beta bits (bit e -> byte e).
__device__ __forceinline__ uint32_t g4(uint32_t a, uint32_t b, uint32_t nib) {
    uint32_t m = ((nib * 0x00204081u) & 0x01010101u) * 0xFFu;
    uint32_t sa = (a & ~m) | (__vneg4(a) & m);
    return __vmaxs4(__vaddss4(b, sa), 0x81818181u);
}

template <int W>
__device__ __forceinline__ void gsync(int gidx) {
    if (W == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(gidx + 1), "n"(W * 32) : "memory");
    }
}

// Buffers live in the group's shared memory or, when spilled, in its global scratch.
template <typename T>
__device__ __forceinline__ T *alpha_ptr(const Layout &lay, uint8_t *S, uint8_t *Gs, int j) {
    return ((lay.spill_mask >> j) & 1u) ? reinterpret_cast<T *>(Gs + lay.galpha[j])
                                        : reinterpret_cast<T *>(S + lay.alpha[j]);
}
__device__ __forceinline__ uint32_t *bl_ptr(const Layout &lay, uint8_t *S, uint8_t *Gs, int j) {
    return ((lay.bl_spill >> j) & 1u) ? reinterpret_cast<uint32_t *>(Gs + lay.gbl[j])
                                      : reinterpret_cast<uint32_t *>(S + lay.bl[j]);
}
__device__ __forceinline__ uint32_t *br_ptr(const Layout &lay, uint8_t *S, uint8_t *Gs) {
    return (lay.flags & LAY_BR_GLOBAL) ? reinterpret_cast<uint32_t *>(Gs + lay.gbr)
                                       : reinterpret_cast<uint32_t *>(S + lay.br);
}
template <typename T>
__device__ __forceinline__ T *chan_ptr(const Layout &lay, uint8_t *S, uint8_t *Gs) {
    return (lay.flags & LAY_CHAN_GLOBAL) ? reinterpret_cast<T *>(Gs + lay.gchan)
                                         : reinterpret_cast<T *>(S + lay.chan);
}

// ---- stages evaluated from the channel (Layout::virt_mask) -----------------
// The top D stages of some codes are not stored: alpha_j of the node holding
// bit s, for path p, is F (Eq. (1)) of alpha_{j+1} when that node is a left
// child, or G (Eq. (2)) with the path's left-sibling beta BL[j] when it is a
// right child, down to the channel row. An F / G reading such a stage
// evaluates its inputs this way (2^D channel loads per element), so those
// stages take no memory. vload4 returns elements 4v .. 4v+3 of alpha_j (f32),
// vload16 elements 16v .. 16v+15 (int8); D = n - j.
template <int D>
__device__ __forceinline__ float4 vload4(const Layout &lay, uint8_t *S, uint8_t *Gs, const float *chan,
                                         const uint8_t *bidxc, int j, int p, int v, uint32_t s) {
    if constexpr (D == 0) {
        return reinterpret_cast<const float4 *>(chan)[v];
    } else {
        const float4 a = vload4<D - 1>(lay, S, Gs, chan, bidxc, j + 1, p, v, s);
        const float4 b = vload4<D - 1>(lay, S, Gs, chan, bidxc, j + 1, p, v + (1 << (j - 2)), s);
        float4 r;
        if ((s >> j) & 1u) {
            const uint32_t *bl = bl_ptr(lay, S, Gs, j) + (int)bidxc[p * 16 + j] * beta_words(j);
            const int i = v << 2;
            const uint32_t nb = bl[i >> 5] >> (i & 31);
            r.x = g_op(a.x, b.x, nb & 1u); r.y = g_op(a.y, b.y, (nb >> 1) & 1u);
            r.z = g_op(a.z, b.z, (nb >> 2) & 1u); r.w = g_op(a.w, b.w, (nb >> 3) & 1u);
        } else {
            r.x = f_op(a.x, b.x); r.y = f_op(a.y, b.y); r.z = f_op(a.z, b.z); r.w = f_op(a.w, b.w);
        }
        return r;
    }
}

template <int D>
__device__ __forceinline__ uint4 vload16(const Layout &lay, uint8_t *S, uint8_t *Gs, const int8_t *chan,
                                         const uint8_t *bidxc, int j, int p, int v, uint32_t s) {
    if constexpr (D == 0) {
        return reinterpret_cast<const uint4 *>(chan)[v];
    } else {
        const uint4 a = vload16<D - 1>(lay, S, Gs, chan, bidxc, j + 1, p, v, s);
        const uint4 b = vload16<D - 1>(lay, S, Gs, chan, bidxc, j + 1, p, v + (1 << (j - 4)), s);
        uint4 r;
        if ((s >> j) & 1u) {
            const uint32_t *bl = bl_ptr(lay, S, Gs, j) + (int)bidxc[p * 16 + j] * beta_words(j);
            const int i = v << 4;
            const uint32_t nb = bl[i >> 5] >> (i & 31);
            r.x = g4(a.x, b.x, nb & 15u); r.y = g4(a.y, b.y, (nb >> 4) & 15u);
            r.z = g4(a.z, b.z, (nb >> 8) & 15u); r.w = g4(a.w, b.w, (nb >> 12) & 15u);
        } else {
            r.x = f4(a.x, b.x); r.y = f4(a.y, b.y); r.z = f4(a.z, b.z); r.w = f4(a.w, b.w);
        }
        return r;
    }
}

// F / G of one node whose input stage j is evaluated from the channel (D =
// n - j levels), writing the stored stage j - 1 for every live path.
template <typename T, int D>
__device__ __noinline__ void fg_virtual(const Layout &lay, uint8_t *S, uint8_t *Gs, const T *chan,
                                           uint8_t *idxc, const uint8_t *bidxc, bool isG, int j, uint32_t s, int La,
                                           int tid, int nthr) {
    const int jo = j - 1;
    const int h = 1 << jo;
    T *outb = alpha_ptr<T>(lay, S, Gs, jo);
    const uint32_t *blb = bl_ptr(lay, S, Gs, jo);
    const int bwc = beta_words(jo);
    if (sizeof(T) == 4) {
        const int lv = jo - 2;
        const int total = La << lv;
        for (int t = tid; t < total; t += nthr) {
            const int p = t >> lv, v = t & ((1 << lv) - 1);
            const float *ch = reinterpret_cast<const float *>(chan);
            const float4 a = vload4<D>(lay, S, Gs, ch, bidxc, j, p, v, s);
            const float4 b = vload4<D>(lay, S, Gs, ch, bidxc, j, p, v + (h >> 2), s);
            float4 r;
            if (isG) {
                const int i = v << 2;
                const uint32_t nb = blb[(int)bidxc[p * 16 + jo] * bwc + (i >> 5)] >> (i & 31);
                r.x = g_op(a.x, b.x, nb & 1u); r.y = g_op(a.y, b.y, (nb >> 1) & 1u);
                r.z = g_op(a.z, b.z, (nb >> 2) & 1u); r.w = g_op(a.w, b.w, (nb >> 3) & 1u);
            } else {
                r.x = f_op(a.x, b.x); r.y = f_op(a.y, b.y); r.z = f_op(a.z, b.z); r.w = f_op(a.w, b.w);
            }
            reinterpret_cast<float4 *>(reinterpret_cast<float *>(outb) + (p << jo))[v] = r;
        }
    } else {
        const int lv = jo - 4;
        const int total = La << lv;
        for (int t = tid; t < total; t += nthr) {
            const int p = t >> lv, v = t & ((1 << lv) - 1);
            const int8_t *ch = reinterpret_cast<const int8_t *>(chan);
            const uint4 a = vload16<D>(lay, S, Gs, ch, bidxc, j, p, v, s);
            const uint4 b = vload16<D>(lay, S, Gs, ch, bidxc, j, p, v + (h >> 4), s);
            uint4 r;
            if (isG) {
                const int i = v << 4;
                const uint32_t nb = blb[(int)bidxc[p * 16 + jo] * bwc + (i >> 5)] >> (i & 31);
                r.x = g4(a.x, b.x, nb & 15u); r.y = g4(a.y, b.y, (nb >> 4) & 15u);
                r.z = g4(a.z, b.z, (nb >> 8) & 15u); r.w = g4(a.w, b.w, (nb >> 12) & 15u);
            } else {
                r.x = f4(a.x, b.x); r.y = f4(a.y, b.y); r.z = f4(a.z, b.z); r.w = f4(a.w, b.w);
            }
            reinterpret_cast<uint4 *>(reinterpret_cast<int8_t *>(outb) + (p << jo))[v] = r;
        }
    }
    for (int t = tid; t < La; t += nthr) idxc[t * 16 + jo] = (uint8_t)t;
}

// SPC candidate flips over the ranks of the four least reliable bits (bit r
// = rank r+1), in the candidate order {}, {1,2}, {1,3}, {1,4}, {2,3}, {2,4},
// {3,4}, {1,2,3,4}.
__device__ __forceinline__ uint32_t spc_tmask(int c) { return (0xFCA69530u >> (4 * c)) & 0xFu; }

// ---- warp-level selection -------------------------------------------------
template <typename K> __device__ __forceinline__ K kmin(K a, K b) { return a < b ? a : b; }
template <typename K> __device__ __forceinline__ K kmax(K a, K b) { return a < b ? b : a; }

template <typename K>
__device__ __forceinline__ K bsort32(K x, int lane) {   // ascending across the warp
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const K o = __shfl_xor_sync(FULL, x, j);
            const bool up = (lane & k) == 0;
            const bool lo = (lane & j) == 0;
            x = (lo == up) ? kmin(x, o) : kmax(x, o);
        }
    }
    return x;
}

template <typename K>
__device__ __forceinline__ K bmerge32(K x, int lane) {  // bitonic -> ascending
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const K o = __shfl_xor_sync(FULL, x, j);
        x = ((lane & j) == 0) ? kmin(x, o) : kmax(x, o);
    }
    return x;
}

template <typename K>
__device__ __forceinline__ void ce(K &a, K &b) {
    const K lo = kmin(a, b), hi = kmax(a, b);
    a = lo;
    b = hi;
}

template <typename K>
__device__ __forceinline__ void sort8(K (&k)[8]) {   // Batcher odd-even merge network
    ce(k[0], k[1]); ce(k[2], k[3]); ce(k[4], k[5]); ce(k[6], k[7]);
    ce(k[0], k[2]); ce(k[1], k[3]); ce(k[4], k[6]); ce(k[5], k[7]);
    ce(k[1], k[2]); ce(k[5], k[6]);
    ce(k[0], k[4]); ce(k[1], k[5]); ce(k[2], k[6]); ce(k[3], k[7]);
    ce(k[2], k[4]); ce(k[3], k[5]);
    ce(k[1], k[2]); ce(k[3], k[4]); ce(k[5], k[6]);
}

__device__ __forceinline__ int warp_excl_scan(int v, int lane) {
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += o;
    }
    return x - v;
}

// The L-th smallest key of the warp, lane s holding its keys sorted in k[]
// (lanes >= La hold none). `tmp` is warp scratch in shared memory for at least
// L keys.
template <typename K>
__device__ __forceinline__ K warp_kth(const K (&k)[8], int C, int L, int La, int lane, K *tmp) {
    if (C >= 4 && La == L) {
        // With a full list, the L sources' best keys are L keys no larger than
        // t0 (the largest of them), so the result is at most t0: only the few
        // later candidates below t0 can still displace a best key.
        K t0 = lane < La ? k[0] : (K)0;
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) t0 = kmax(t0, __shfl_xor_sync(FULL, t0, m));
        int t = 0;
#pragma unroll
        for (int r = 1; r < 8; ++r) t += k[r] < t0 ? 1 : 0;
        const int base = warp_excl_scan(t, lane);
        const int tot = __shfl_sync(FULL, base + t, 31);
        if (tot == 0) return t0;
        if (tot <= 3) {
            // few extra keys: the result is the (tot + 1)-th largest of the L
            // best keys and the extras; take the largest tot times away
            if (t > 0) {
#pragma unroll
                for (int r = 1; r < 8; ++r)
                    if (r <= t) tmp[base + r - 1] = k[r];
            }
            __syncwarp();
            K c0 = lane < La ? k[0] : (K)0;
            K c1 = lane < tot ? tmp[lane] : (K)0;
            __syncwarp();
            for (int r = 0;; ++r) {
                K m = kmax(c0, c1);
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) m = kmax(m, __shfl_xor_sync(FULL, m, d));
                if (r == tot) return m;
                if (c0 == m) c0 = (K)0;
                else if (c1 == m) c1 = (K)0;
            }
        }
        if (tot <= L) {
#pragma unroll
            for (int r = 1; r < 8; ++r)
                if (r <= t) tmp[base + r - 1] = k[r];
            __syncwarp();
            K y = lane < tot ? tmp[lane] : ~(K)0;
            __syncwarp();
            K B = bsort32(k[0], lane);
            y = bsort32(y, lane);
            y = __shfl_sync(FULL, y, 31 - lane);      // descending
            B = bmerge32(kmin(B, y), lane);
            return __shfl_sync(FULL, B, L - 1);
        }
    }
    // General case: column r (every lane's r-th key) can change the result
    // only while its minimum is below the current L-th key; each lane's
    // columns only grow.
    K B = bsort32(k[0], lane);
    K tau = __shfl_sync(FULL, B, L - 1);
    // later columns, one per iteration (kept rolled: the body is large)
    K q[7];
#pragma unroll
    for (int r = 0; r < 7; ++r) q[r] = k[r + 1];
#pragma unroll 1
    for (int r = 1; r < C; ++r) {
        K col = q[0];
#pragma unroll
        for (int t = 0; t < 6; ++t) q[t] = q[t + 1];
        K mn = col;
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) mn = kmin(mn, __shfl_xor_sync(FULL, mn, m));
        if (mn > tau) break;
        col = bsort32(col, lane);
        col = __shfl_sync(FULL, col, 31 - lane);      // descending
        B = bmerge32(kmin(B, col), lane);
        tau = __shfl_sync(FULL, B, L - 1);
    }
    return tau;
}

// ---- segmented selection: several frames' paths in one warp ----------------
// With L <= 16 paths a warp holds P = 32 / L frames' subtrees at once: lane
// sb + s is path s of the frame whose segment starts at lane sb, and every
// sort, scan and reduction stays inside an aligned segment of sn = L lanes
// (xor partners below sn never leave it). Branches that depend on the data of
// one segment are taken warp-uniformly (on the warp's maximum), so every
// shuffle sees the whole warp.
template <typename K>
__device__ __forceinline__ K bsort_seg(K x, int ls, int sn) {   // ascending inside each segment
    for (int k = 2; k <= sn; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const K o = __shfl_xor_sync(FULL, x, j);
            const bool up = (ls & k) == 0;
            const bool lo = (ls & j) == 0;
            x = (lo == up) ? kmin(x, o) : kmax(x, o);
        }
    }
    return x;
}

template <typename K>
__device__ __forceinline__ K bmerge_seg(K x, int ls, int sn) {  // bitonic -> ascending inside each segment
    for (int j = sn >> 1; j > 0; j >>= 1) {
        const K o = __shfl_xor_sync(FULL, x, j);
        x = ((ls & j) == 0) ? kmin(x, o) : kmax(x, o);
    }
    return x;
}

__device__ __forceinline__ int seg_excl_scan(int v, int ls, int sn) {
    int x = v;
    for (int d = 1; d < sn; d <<= 1) {
        const int o = __shfl_up_sync(FULL, x, d);
        if (ls >= d) x += o;
    }
    return x - v;
}

template <typename K>
__device__ __forceinline__ K seg_max(K x, int sn) {
    for (int m = sn >> 1; m > 0; m >>= 1) x = kmax(x, __shfl_xor_sync(FULL, x, m));
    return x;
}
template <typename K>
__device__ __forceinline__ K seg_min(K x, int sn) {
    for (int m = sn >> 1; m > 0; m >>= 1) x = kmin(x, __shfl_xor_sync(FULL, x, m));
    return x;
}

// warp_kth for segments of sn = L lanes (tmp: the segment's frame's scratch).
template <typename K>
__device__ __forceinline__ K warp_kth_seg(const K (&k)[8], int C, int L, int La, int sb, int ls, K *tmp) {
    const int sn = L;
    if (C >= 4 && La == L) {
        const K t0 = seg_max<K>(k[0], sn);
        int t = 0;
#pragma unroll
        for (int r = 1; r < 8; ++r) t += k[r] < t0 ? 1 : 0;
        const int base = seg_excl_scan(t, ls, sn);
        const int tot = __shfl_sync(FULL, base + t, sb + sn - 1);
        int tmax = tot;
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) tmax = max(tmax, __shfl_xor_sync(FULL, tmax, m));
        if (tmax == 0) return t0;
        if (tmax <= 3 && tmax <= sn) {      // one extra key per lane of the segment
            if (t > 0) {
#pragma unroll
                for (int r = 1; r < 8; ++r)
                    if (r <= t) tmp[base + r - 1] = k[r];
            }
            __syncwarp();
            K c0 = k[0];
            K c1 = ls < tot ? tmp[ls] : (K)0;
            __syncwarp();
            K res = t0;
            for (int r = 0; r <= tmax; ++r) {
                const K m = seg_max<K>(kmax(c0, c1), sn);
                if (r == tot) res = m;
                if (c0 == m) c0 = (K)0;
                else if (c1 == m) c1 = (K)0;
            }
            return res;
        }
        if (tmax <= L) {
#pragma unroll
            for (int r = 1; r < 8; ++r)
                if (r <= t) tmp[base + r - 1] = k[r];
            __syncwarp();
            K y = ls < tot ? tmp[ls] : ~(K)0;
            __syncwarp();
            K B = bsort_seg(k[0], ls, sn);
            y = bsort_seg(y, ls, sn);
            y = __shfl_sync(FULL, y, sb + sn - 1 - ls);      // descending
            B = bmerge_seg(kmin(B, y), ls, sn);
            return __shfl_sync(FULL, B, sb + L - 1);
        }
    }
    K B = bsort_seg(k[0], ls, sn);
    K tau = __shfl_sync(FULL, B, sb + L - 1);
    K q[7];
#pragma unroll
    for (int r = 0; r < 7; ++r) q[r] = k[r + 1];
#pragma unroll 1
    for (int r = 1; r < C; ++r) {
        K col = q[0];
#pragma unroll
        for (int t = 0; t < 6; ++t) q[t] = q[t + 1];
        const K mn = seg_min<K>(col, sn);
        // a column above every segment's threshold changes no segment (merging it
        // into one below its threshold would not either)
        if (__all_sync(FULL, mn > tau)) break;
        col = bsort_seg(col, ls, sn);
        col = __shfl_sync(FULL, col, sb + sn - 1 - ls);      // descending
        B = bmerge_seg(kmin(B, col), ls, sn);
        tau = __shfl_sync(FULL, B, sb + L - 1);
    }
    return tau;
}

template <typename KT>
__device__ __noinline__ KT select_keys_seg(KT k0, KT k1, KT k2, KT k3, KT k4, KT k5, KT k6, KT k7, int C, int nc,
                                           int L, int sb, int ls, KT *tab) {
    const KT KINF = (KT)~(KT)0;
    KT k[8] = {k0, k1, k2, k3, k4, k5, k6, k7};
    const KT tau = (nc > L) ? warp_kth_seg(k, C, L, nc / C, sb, ls, tab) : KINF;
    const uint32_t cm = (uint32_t)(C - 1);
    uint32_t sm = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r)
        if (k[r] != KINF && k[r] <= tau) sm |= 1u << ((uint32_t)k[r] & cm);
    const int base = seg_excl_scan(__popc(sm), ls, L);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        if (k[r] != KINF && k[r] <= tau) tab[base + __popc(sm & ((1u << ((uint32_t)k[r] & cm)) - 1u))] = k[r];
    }
    __syncwarp();
    const int La2 = nc < L ? nc : L;
    return ls < La2 ? tab[ls] : (KT)0;
}

// ---- register-resident subtrees (OP_SUB) ----------------------------------
// A subtree of at most 16 bits runs on warp 0, lane s = path s. The alpha of
// stage j (j <= 4) lives in registers a[(1 << j) - 1 ...], left-child betas in
// bl[j], the latest right-child beta in br. A fork moves a path's live state
// (alpha of the stages above the leaf, pending left betas, penalty, origin)
// from its parent lane with warp shuffles.
template <int J> __device__ __forceinline__ constexpr int aoff() { return (1 << J) - 1; }

__device__ __forceinline__ float fv(float a, float b) { return f_op(a, b); }
__device__ __forceinline__ int fv(int a, int b) {
    const int m = min(abs(a), abs(b));
    return ((a ^ b) < 0) ? -m : m;
}
__device__ __forceinline__ float gv(float a, float b, uint32_t beta) { return g_op(a, b, beta); }
__device__ __forceinline__ int gv(int a, int b, uint32_t beta) {
    const int r = beta ? b - a : b + a;
    return max(-127, min(127, r));
}

template <typename T>
struct Sub {
    typedef typename Arith<T>::P P;
    P a[31];
    uint32_t bl[5];
    uint32_t br;
    P pen;
    int orig;
};

template <typename T>
struct SubCtx {
    typename Arith<T>::K *tab;     // survivor keys in new-slot order (shared memory)
    int lane, La, L;
    bool live;                     // the lane's segment holds a frame (segmented mode)
};

struct Desc {
    unsigned long long w0, w1;
    int pos;
    __device__ __forceinline__ uint32_t next() {
        const uint32_t v = pos < 21 ? (uint32_t)(w0 >> (3 * pos)) & 7u : (uint32_t)(w1 >> (3 * (pos - 21))) & 7u;
        ++pos;
        return v;
    }
};

// Selection (Algorithm 1) for lane-per-path leaves: keep the L smallest keys,
// survivors renumbered in (source, candidate) order; returns lane t's new key.
template <typename KT>
__device__ __noinline__ KT select_keys(KT k0, KT k1, KT k2, KT k3, KT k4, KT k5, KT k6, KT k7, int C, int nc, int L,
                                       int lane, KT *tab) {
    const KT KINF = (KT)~(KT)0;
    KT k[8] = {k0, k1, k2, k3, k4, k5, k6, k7};
    const KT tau = (nc > L) ? warp_kth(k, C, L, nc / C, lane, tab) : KINF;
    const uint32_t cm = (uint32_t)(C - 1);
    uint32_t sm = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r)
        if (k[r] != KINF && k[r] <= tau) sm |= 1u << ((uint32_t)k[r] & cm);
    const int base = warp_excl_scan(__popc(sm), lane);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        if (k[r] != KINF && k[r] <= tau) tab[base + __popc(sm & ((1u << ((uint32_t)k[r] & cm)) - 1u))] = k[r];
    }
    __syncwarp();
    const int La2 = nc < L ? nc : L;
    return lane < La2 ? tab[lane] : (KT)0;
}

template <typename T, int J, bool SEGD>
__device__ __forceinline__ void sub_leaf(uint32_t type, Sub<T> &st, int side, SubCtx<T> &cx) {
    typedef typename Arith<T>::P P;
    typedef typename Arith<T>::K KT;
    constexpr KT KINF = Arith<T>::KINF;
    constexpr int nv = 1 << J;
    constexpr int o = aoff<J>();
    constexpr uint32_t wmask = (nv >= 32) ? 0xffffffffu : ((1u << nv) - 1u);
    const int lane = cx.lane;
    // path index inside the frame and first lane of the frame (packed frames: segments of L lanes)
    const int ls = SEGD ? (lane & (cx.L - 1)) : lane;
    const int sb = SEGD ? (lane & ~(cx.L - 1)) : 0;
    const bool live = SEGD ? cx.live : true;
    const bool act = live && ls < cx.La;
    if (type == OP_R0) {
        // Rate-0 (Sec. III-B): penalty += sum |min(a, 0)| (pairwise tree), beta = 0.
        P x[nv];
#pragma unroll
        for (int i = 0; i < nv; ++i) x[i] = Arith<T>::negpart(st.a[o + i]);
#pragma unroll
        for (int h = nv >> 1; h >= 1; h >>= 1)
#pragma unroll
            for (int i = 0; i < h; ++i) x[i] = x[i] + x[i + h];
        if (act) st.pen = st.pen + x[0];
        if (side) st.br = 0u; else st.bl[J] = 0u;
        return;
    }
    uint32_t hd = 0;
#pragma unroll
    for (int i = 0; i < nv; ++i)
        if (st.a[o + i] < 0) hd |= 1u << i;
    KT k[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) k[c] = KINF;
    uint32_t mpos = 0, flag = 0;
    int C, lc;
    const int s = ls;
    const P ps = st.pen;
    // a leaf of one bit is Rate-0 or Rate-1; SPC needs at least four bits
    if (J >= 1 && type == OP_REP) {
        // Repetition (Sec. III-E): the ML word listed first.
        C = 2;
        lc = 1;
        P x0[nv], x1[nv];
#pragma unroll
        for (int i = 0; i < nv; ++i) {
            x0[i] = Arith<T>::negpart(st.a[o + i]);
            x1[i] = Arith<T>::pospart(st.a[o + i]);
        }
#pragma unroll
        for (int h = nv >> 1; h >= 1; h >>= 1)
#pragma unroll
            for (int i = 0; i < h; ++i) {
                x0[i] = x0[i] + x0[i + h];
                x1[i] = x1[i] + x1[i + h];
            }
        flag = (x0[0] <= x1[0]) ? 0u : 1u;
        k[0] = Arith<T>::mk(ps + (flag ? x1[0] : x0[0]), s * 2 + 0);
        k[1] = Arith<T>::mk(ps + (flag ? x0[0] : x1[0]), s * 2 + 1);
    } else {
        // least reliable positions by (|a|, index): keys |a| << 4 | i (32 bits hold them for int8)
        typedef typename std::conditional<sizeof(T) == 1, uint32_t, unsigned long long>::type LKT;
        LKT lk[4] = {~(LKT)0, ~(LKT)0, ~(LKT)0, ~(LKT)0};
        if (nv <= 4) {
            // a sorting network over the (at most four) keys
#pragma unroll
            for (int i = 0; i < nv; ++i) lk[i] = ((LKT)Arith<T>::absbits(st.a[o + i]) << 4) | (unsigned)i;
            if (nv >= 2) ce(lk[0], lk[1]);
            if (nv == 4) {
                ce(lk[2], lk[3]); ce(lk[0], lk[2]); ce(lk[1], lk[3]); ce(lk[1], lk[2]);
            }
        } else {
            // R passes of a plain minimum over the keys not taken yet
            const int R = (J < 2 || type == OP_R1) ? 2 : 4;
#pragma unroll 1
            for (int r = 0; r < R; ++r) {
                const LKT prev = r > 0 ? lk[r - 1] : (LKT)0;
                LKT best = ~(LKT)0;
#pragma unroll
                for (int i = 0; i < nv; ++i) {
                    const LKT v = ((LKT)Arith<T>::absbits(st.a[o + i]) << 4) | (unsigned)i;
                    if ((r == 0 || v > prev) && v < best) best = v;
                }
                if (r == 0) lk[0] = best; else if (r == 1) lk[1] = best; else if (r == 2) lk[2] = best; else lk[3] = best;
            }
        }
        P ar[4];
        uint32_t m[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            ar[r] = Arith<T>::unabs((uint32_t)(lk[r] >> 4));
            m[r] = (uint32_t)(lk[r] & 15u);
        }
        mpos = m[0] | (m[1] << 4) | (m[2] << 8) | (m[3] << 12);
        if (J < 2 || type == OP_R1) {
            // Rate-1 (Sec. III-C): HD, HD^m1, HD^m2, HD^m1^m2.
            C = nv == 1 ? 2 : 4;
            lc = nv == 1 ? 1 : 2;
            k[0] = Arith<T>::mk(ps, s * C + 0);
            k[1] = Arith<T>::mk(ps + ar[0], s * C + 1);
            if (nv > 1) {
                k[2] = Arith<T>::mk(ps + ar[1], s * C + 2);
                k[3] = Arith<T>::mk(ps + (ar[0] + ar[1]), s * C + 3);
            }
        } else {
            // SPC (Sec. III-D): ML = HD or HD^m1; ML ^ T, penalty from Eq. (9).
            C = cx.L == 2 ? 2 : 8;
            lc = cx.L == 2 ? 1 : 3;
            flag = (__popc(hd) & 1u) ? 0u : 1u;   // q
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (c < C) {
                    const uint32_t dm = spc_tmask(c) ^ (flag ? 0u : 1u);
                    P inc = (P)0;
                    bool first = true;
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if ((dm >> r) & 1u) { inc = first ? ar[r] : inc + ar[r]; first = false; }
                    k[c] = Arith<T>::mk(ps + inc, s * C + c);
                }
            }
            if (C == 8) sort8(k);
        }
    }
    if (!act) {
#pragma unroll
        for (int c = 0; c < 8; ++c) k[c] = KINF;
    }
    const int nc = cx.La * C;
    const KT kt = SEGD ? select_keys_seg<KT>(k[0], k[1], k[2], k[3], k[4], k[5], k[6], k[7], C, nc, cx.L, sb, ls, cx.tab)
                       : select_keys<KT>(k[0], k[1], k[2], k[3], k[4], k[5], k[6], k[7], C, nc, cx.L, lane, cx.tab);
    const int La2 = nc < cx.L ? nc : cx.L;
    const bool act2 = live && ls < La2;
    const uint32_t ci = Arith<T>::kidx(kt);
    const int src = sb + (act2 ? (int)(ci >> lc) : 0);
    const int c = (int)(ci & (uint32_t)(C - 1));
    const uint32_t hd_s = __shfl_sync(FULL, hd, src);
    const uint32_t mp_s = __shfl_sync(FULL, mpos, src);
    const uint32_t fl_s = __shfl_sync(FULL, flag, src);
#pragma unroll
    for (int i = o + nv; i < 31; ++i) st.a[i] = __shfl_sync(FULL, st.a[i], src);
#pragma unroll
    for (int jj = J; jj < 5; ++jj) st.bl[jj] = __shfl_sync(FULL, st.bl[jj], src);
    st.orig = __shfl_sync(FULL, st.orig, src);
    if (act2) st.pen = Arith<T>::kpen(kt);
    uint32_t word;
    if (J >= 1 && type == OP_REP) {
        word = ((fl_s != 0u) != (c == 1)) ? wmask : 0u;
    } else {
        const uint32_t dm = (J < 2 || type == OP_R1) ? (uint32_t)c : (spc_tmask(c) ^ (fl_s ? 0u : 1u));
        word = hd_s;
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
            if ((dm >> rr) & 1u) word ^= 1u << ((mp_s >> (4 * rr)) & 15u);
    }
    if (side) st.br = word; else st.bl[J] = word;
    cx.La = La2;
    __syncwarp();
}

template <typename T, int J, bool SEGD>
__device__ __forceinline__ void sub_node(Sub<T> &st, Desc &d, int side, SubCtx<T> &cx) {
    const uint32_t type = d.next();
    if (J == 0 || type != 0u) {
        sub_leaf<T, J, SEGD>(type, st, side, cx);
        return;
    }
    if constexpr (J > 0) {
        constexpr int h = 1 << (J - 1);
#pragma unroll 1
        for (int sd = 0; sd < 2; ++sd) {
            if (sd == 0) {
#pragma unroll
                for (int i = 0; i < h; ++i) st.a[aoff<J - 1>() + i] = fv(st.a[aoff<J>() + i], st.a[aoff<J>() + i + h]);
            } else {
#pragma unroll
                for (int i = 0; i < h; ++i)
                    st.a[aoff<J - 1>() + i] =
                        gv(st.a[aoff<J>() + i], st.a[aoff<J>() + i + h], (st.bl[J - 1] >> i) & 1u);
            }
            sub_node<T, J - 1, SEGD>(st, d, sd, cx);
        }
        constexpr uint32_t m = (1u << h) - 1u;
        const uint32_t v = ((st.bl[J - 1] ^ st.br) & m) | ((st.br & m) << h);
        if (side == 0) st.bl[J] = v; else st.br = v;
    }
}

// ---- run one register subtree -------------------------------------------
// Warp 0: load the paths' alpha rows of stage JR, walk the subtree, then write
// the root's beta, penalties and index rows. With SEGD the warp holds
// 32 / L frames of L paths each (lane f * L + s = path s of frame f, whose
// memory starts sstride bytes of shared memory and gstride bytes of scratch
// after frame f - 1's).
template <typename T, int JR, bool SEGD>
__device__ __forceinline__ void run_sub(const CodeView &cv, uint8_t *S, uint8_t *Gs, uint32_t op, int La, int cur,
                                        int lane, int P = 1, uint32_t sstride = 0, uint64_t gstride = 0) {
    typedef typename Arith<T>::P PT;
    typedef typename Arith<T>::K KT;
    const Layout &lay = cv.lay;
    const int me = SEGD ? (lane & (cv.L - 1)) : lane;           // path index inside the frame
    const int fseg = SEGD ? lane / cv.L : 0;                     // the lane's frame (segment)
    const bool live = fseg < P;                                  // segments past the P frames idle
    if (SEGD && live) {
        S += (size_t)fseg * sstride;
        if (Gs) Gs += (size_t)fseg * gstride;
    }
    const int n = cv.n;
    const int dest = op_dest(op);
    uint8_t *idxc = S + lay.idx[cur];
    uint8_t *bidxc = S + lay.bidx[cur];
    PT *penc = reinterpret_cast<PT *>(S + lay.pen[cur]);
    Sub<T> st;
    const bool act = live && me < La;
    const T *row = (JR == n) ? chan_ptr<T>(lay, S, Gs)
                             : alpha_ptr<T>(lay, S, Gs, JR) + ((int)idxc[(act ? me : 0) * 16 + JR] << JR);
    constexpr int o = aoff<JR>();
#pragma unroll
    for (int i = 0; i < 31; ++i) st.a[i] = 0;
    if (act) {
        if (sizeof(T) == 4) {
#pragma unroll
            for (int q = 0; q < (1 << JR) / 4; ++q) {
                const float4 v = reinterpret_cast<const float4 *>(row)[q];
                st.a[o + 4 * q] = v.x; st.a[o + 4 * q + 1] = v.y; st.a[o + 4 * q + 2] = v.z; st.a[o + 4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < (1 << JR) / 4; ++q) {
                const uint32_t v = reinterpret_cast<const uint32_t *>(row)[q];
                st.a[o + 4 * q] = (int)(int8_t)(v & 0xFF);
                st.a[o + 4 * q + 1] = (int)(int8_t)((v >> 8) & 0xFF);
                st.a[o + 4 * q + 2] = (int)(int8_t)((v >> 16) & 0xFF);
                st.a[o + 4 * q + 3] = (int)(int8_t)(v >> 24);
            }
        }
        st.pen = penc[me];
    } else {
        st.pen = (PT)0;
    }
#pragma unroll
    for (int jj = 0; jj < 5; ++jj) st.bl[jj] = 0u;
    st.br = 0u;
    st.orig = me;
    const uint32_t di = op_sub_desc(op);
    Desc d;
    d.w0 = __ldg(cv.desc + 2 * di);
    d.w1 = __ldg(cv.desc + 2 * di + 1);
    d.pos = 0;
    SubCtx<T> cx;
    cx.tab = reinterpret_cast<KT *>(S + lay.surv);
    cx.lane = lane;
    cx.La = La;
    cx.L = cv.L;
    cx.live = live;
    sub_node<T, JR, SEGD>(st, d, dest, cx);
    const bool act2 = live && me < cx.La;
    const uint32_t beta = dest ? st.br : st.bl[JR];
    uint32_t *bout = dest ? br_ptr(lay, S, Gs) : bl_ptr(lay, S, Gs, JR);
    const int ostride = dest ? beta_words(n) : beta_words(JR);
    if (act2) {
        if (op_sub_fork(op)) {
            const int nxt = cur ^ 1;
            uint8_t *idxn = S + lay.idx[nxt];
            uint8_t *bidxn = S + lay.bidx[nxt];
            reinterpret_cast<PT *>(S + lay.pen[nxt])[me] = st.pen;
            reinterpret_cast<uint4 *>(idxn)[me] = reinterpret_cast<const uint4 *>(idxc)[st.orig];
            reinterpret_cast<uint4 *>(bidxn)[me] = reinterpret_cast<const uint4 *>(bidxc)[st.orig];
            if (!dest) bidxn[me * 16 + JR] = (uint8_t)me;
        } else {
            penc[me] = st.pen;
            if (!dest) bidxc[me * 16 + JR] = (uint8_t)me;
        }
        bout[me * ostride] = beta;
    }
}

// ---- one inner node of 32 bits as a single operation ----------------------
// F (Eq. (1)), the left register subtree, G (Eq. (2)), the right register
// subtree and Combine (Eq. (3)) of a node just above the register subtrees,
// on warp 0 with lane s = path s. The node's input row stays in memory and is
// read twice, the second time through the row index of the path the lane
// descends from (st.orig), so stage-4 rows and left betas never leave
// registers.
template <typename T>
__device__ __forceinline__ void node32_in(const T *row, Sub<T> &st, int side) {
    constexpr int o = aoff<kSubLog>();
    if (sizeof(T) == 4) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 x = r4[q], y = r4[q + 4];
            const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = 4 * q + e;
                st.a[o + i] = side ? gv(xs[e], ys[e], (st.bl[kSubLog] >> i) & 1u) : fv(xs[e], ys[e]);
            }
        }
    } else {
        const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
        const uint4 x4 = r4[0], y4 = r4[1];
        const uint32_t xw[4] = {x4.x, x4.y, x4.z, x4.w}, yw[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int a = (int)(int8_t)((xw[i >> 2] >> (8 * (i & 3))) & 0xFF);
            const int b = (int)(int8_t)((yw[i >> 2] >> (8 * (i & 3))) & 0xFF);
            st.a[o + i] = side ? gv(a, b, (st.bl[kSubLog] >> i) & 1u) : fv(a, b);
        }
    }
}

template <typename T, bool SEGD>
__device__ __forceinline__ void run_sub32(const CodeView &cv, uint8_t *S, uint8_t *Gs, uint32_t op, int La, int cur,
                                          int lane, int P = 1, uint32_t sstride = 0, uint64_t gstride = 0) {
    typedef typename Arith<T>::P PT;
    typedef typename Arith<T>::K KT;
    constexpr int JN = kSubLog + 1;
    const Layout &lay = cv.lay;
    const int me = SEGD ? (lane & (cv.L - 1)) : lane;           // path index inside the frame
    const int fseg = SEGD ? lane / cv.L : 0;                     // the lane's frame (segment)
    const bool live = fseg < P;                                  // segments past the P frames idle
    if (SEGD && live) {
        S += (size_t)fseg * sstride;
        if (Gs) Gs += (size_t)fseg * gstride;
    }
    const int n = cv.n;
    const int dest = op_dest(op);
    uint8_t *idxc = S + lay.idx[cur];
    uint8_t *bidxc = S + lay.bidx[cur];
    PT *penc = reinterpret_cast<PT *>(S + lay.pen[cur]);
    const T *stj = alpha_ptr<T>(lay, S, Gs, JN);
    Sub<T> st;
#pragma unroll
    for (int i = 0; i < 31; ++i) st.a[i] = 0;
    st.pen = (live && me < La) ? penc[me] : (PT)0;
#pragma unroll
    for (int jj = 0; jj < 5; ++jj) st.bl[jj] = 0u;
    st.br = 0u;
    st.orig = me;
    SubCtx<T> cx;
    cx.tab = reinterpret_cast<KT *>(S + lay.surv);
    cx.lane = lane;
    cx.La = La;
    cx.L = cv.L;
    cx.live = live;
    const uint32_t di = op_sub_desc(op);
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        if (live && me < cx.La) node32_in<T>(stj + ((int)idxc[st.orig * 16 + JN] << JN), st, side);
        Desc d;
        d.w0 = __ldg(cv.desc + 2 * (di + side));
        d.w1 = __ldg(cv.desc + 2 * (di + side) + 1);
        d.pos = 0;
        sub_node<T, kSubLog, SEGD>(st, d, side, cx);
    }
    const bool act2 = live && me < cx.La;
    const uint32_t beta = ((st.bl[kSubLog] ^ st.br) & 0xFFFFu) | ((st.br & 0xFFFFu) << 16);
    uint32_t *bout = dest ? br_ptr(lay, S, Gs) : bl_ptr(lay, S, Gs, JN);
    const int ostride = dest ? beta_words(n) : beta_words(JN);
    if (act2) {
        if (op_sub_fork(op)) {
            const int nxt = cur ^ 1;
            uint8_t *idxn = S + lay.idx[nxt];
            uint8_t *bidxn = S + lay.bidx[nxt];
            reinterpret_cast<PT *>(S + lay.pen[nxt])[me] = st.pen;
            reinterpret_cast<uint4 *>(idxn)[me] = reinterpret_cast<const uint4 *>(idxc)[st.orig];
            reinterpret_cast<uint4 *>(bidxn)[me] = reinterpret_cast<const uint4 *>(bidxc)[st.orig];
            if (!dest) bidxn[me * 16 + JN] = (uint8_t)me;
        } else {
            penc[me] = st.pen;
            if (!dest) bidxc[me * 16 + JN] = (uint8_t)me;
        }
        bout[me * ostride] = beta;
    }
}

// ---- large leaves (more than 16 bits), warp 0, lane s = source path s ----

// Canonical sums of |min(a,0)| (v0) and |max(a,0)| (v1) over one row of nv
// (>= 32) elements. float: the pairwise tree s[i] = x[i] + x[i + n/2] is
// evaluated in place on the row (the leaf input is dead afterwards); int8:
// exact integer sums.
template <typename T>
__device__ __forceinline__ void lane_sums(T *row, int nv, bool want1, typename Arith<T>::P &v0,
                                          typename Arith<T>::P &v1) {
    if (sizeof(T) == 4) {
        float *x = reinterpret_cast<float *>(row);
        const int h = nv >> 1;
        for (int i = 0; i < h; i += 4) {
            const float4 a = *reinterpret_cast<const float4 *>(x + i);
            const float4 b = *reinterpret_cast<const float4 *>(x + h + i);
            float4 y0, y1;
            y0.x = Arith<float>::negpart(a.x) + Arith<float>::negpart(b.x);
            y0.y = Arith<float>::negpart(a.y) + Arith<float>::negpart(b.y);
            y0.z = Arith<float>::negpart(a.z) + Arith<float>::negpart(b.z);
            y0.w = Arith<float>::negpart(a.w) + Arith<float>::negpart(b.w);
            *reinterpret_cast<float4 *>(x + i) = y0;
            if (want1) {
                y1.x = Arith<float>::pospart(a.x) + Arith<float>::pospart(b.x);
                y1.y = Arith<float>::pospart(a.y) + Arith<float>::pospart(b.y);
                y1.z = Arith<float>::pospart(a.z) + Arith<float>::pospart(b.z);
                y1.w = Arith<float>::pospart(a.w) + Arith<float>::pospart(b.w);
                *reinterpret_cast<float4 *>(x + h + i) = y1;
            }
        }
        for (int hh = h >> 1; hh >= 1; hh >>= 1) {
            if (hh >= 4) {
                for (int i = 0; i < hh; i += 4) {
                    float4 a = *reinterpret_cast<const float4 *>(x + i);
                    const float4 b = *reinterpret_cast<const float4 *>(x + hh + i);
                    a.x = a.x + b.x; a.y = a.y + b.y; a.z = a.z + b.z; a.w = a.w + b.w;
                    *reinterpret_cast<float4 *>(x + i) = a;
                    if (want1) {
                        float4 c = *reinterpret_cast<const float4 *>(x + h + i);
                        const float4 d = *reinterpret_cast<const float4 *>(x + h + hh + i);
                        c.x = c.x + d.x; c.y = c.y + d.y; c.z = c.z + d.z; c.w = c.w + d.w;
                        *reinterpret_cast<float4 *>(x + h + i) = c;
                    }
                }
            } else {
                for (int i = 0; i < hh; ++i) {
                    x[i] = x[i] + x[i + hh];
                    if (want1) x[h + i] = x[h + i] + x[h + i + hh];
                }
            }
        }
        v0 = (typename Arith<T>::P)x[0];
        v1 = want1 ? (typename Arith<T>::P)x[h] : (typename Arith<T>::P)0;
    } else {
        int s0 = 0, s1 = 0;
        const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
        for (int q = 0; q < (nv >> 4); ++q) {
            const uint4 v = r4[q];
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int a = (int)(int8_t)((w[e] >> (8 * b)) & 0xFF);
                    s0 += a < 0 ? -a : 0;
                    s1 += a > 0 ? a : 0;
                }
            }
        }
        v0 = (typename Arith<T>::P)s0;
        v1 = (typename Arith<T>::P)s1;
    }
}

// Least-reliable-bit keys: |a| << 12 | position (float: 64-bit, int8: 32-bit).
template <typename T> struct LrbKey;
template <> struct LrbKey<float> {
    typedef unsigned long long K;
    static __device__ __forceinline__ K make(float a, int pos) {
        return ((K)__float_as_uint(fabsf(a)) << 12) | (unsigned)pos;
    }
};
template <> struct LrbKey<int8_t> {
    typedef uint32_t K;
    static __device__ __forceinline__ K make(int a, int pos) { return ((uint32_t)(a < 0 ? -a : a) << 12) | (unsigned)pos; }
};

template <typename K, int R>
__device__ __forceinline__ void lrb_insert(K (&top)[4], K v) {
    if (v < top[R - 1]) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (v < top[r]) { const K t = top[r]; top[r] = v; v = t; }
        }
    }
}

// One scan of a row: the R least reliable positions and the number of negative LLRs.
template <typename T, int R>
__device__ __forceinline__ void lane_lrb(const T *row, int nv, typename LrbKey<T>::K (&top)[4], int &neg) {
    typedef typename LrbKey<T>::K K;
#pragma unroll
    for (int r = 0; r < 4; ++r) top[r] = (K)~(K)0;
    int cnt = 0;
    if (sizeof(T) == 4) {
        const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll 4
        for (int q = 0; q < (nv >> 2); ++q) {
            const float4 v = r4[q];
            cnt += (v.x < 0.f) + (v.y < 0.f) + (v.z < 0.f) + (v.w < 0.f);
            lrb_insert<K, R>(top, LrbKey<T>::make(v.x, 4 * q));
            lrb_insert<K, R>(top, LrbKey<T>::make(v.y, 4 * q + 1));
            lrb_insert<K, R>(top, LrbKey<T>::make(v.z, 4 * q + 2));
            lrb_insert<K, R>(top, LrbKey<T>::make(v.w, 4 * q + 3));
        }
    } else {
        const uint4 *r4 = reinterpret_cast<const uint4 *>(row);
        for (int q = 0; q < (nv >> 4); ++q) {
            const uint4 v = r4[q];
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                cnt += __popc(w[e] & 0x80808080u);
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    lrb_insert<K, R>(top, LrbKey<T>::make((int)(int8_t)((w[e] >> (8 * b)) & 0xFF), 16 * q + 4 * e + b));
            }
        }
    }
    neg = cnt;
}

// Hard decisions of 32 consecutive LLRs as one word (bit i <-> element i).
template <typename T>
__device__ __forceinline__ uint32_t hd_word(const T *p) {
    uint32_t w = 0;
    if (sizeof(T) == 4) {
        const float4 *r4 = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 v = r4[q];
            w |= ((uint32_t)(v.x < 0.f) | ((uint32_t)(v.y < 0.f) << 1) | ((uint32_t)(v.z < 0.f) << 2) |
                  ((uint32_t)(v.w < 0.f) << 3)) << (4 * q);
        }
    } else {
        const uint4 *r4 = reinterpret_cast<const uint4 *>(p);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint4 v = r4[h];
            const uint32_t x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const uint32_t t = (x[e] >> 7) & 0x01010101u;              // sign bit of each byte
                w |= (((t * 0x01020408u) >> 24) & 0xFu) << (16 * h + 4 * e);
            }
        }
    }
    return w;
}

template <typename T, bool SEG>
__device__ __forceinline__ void big_leaf(const CodeView &cv, uint8_t *S, uint8_t *Gs, uint32_t kind, int j, int dest,
                                         int La, int cur, int lane) {
    typedef typename Arith<T>::P PT;
    typedef typename Arith<T>::K KT;
    typedef typename LrbKey<T>::K LK;
    constexpr KT KINF = Arith<T>::KINF;
    const Layout &lay = cv.lay;
    const int n = cv.n, L = cv.L;
    const int nv = 1 << j;
    const int bw = nv >> 5;
    T *stj = (j == n) ? chan_ptr<T>(lay, S, Gs) : alpha_ptr<T>(lay, S, Gs, j);
    uint8_t *idxc = S + lay.idx[cur];
    uint8_t *bidxc = S + lay.bidx[cur];
    PT *penc = reinterpret_cast<PT *>(S + lay.pen[cur]);
    uint32_t *bout = dest ? br_ptr(lay, S, Gs) : bl_ptr(lay, S, Gs, j);
    const int ostride = dest ? beta_words(n) : bw;
    const bool act = lane < La;
    const int s = lane;
    T *row = stj + (j == n ? 0 : ((int)idxc[(act ? s : 0) * 16 + j] << j));
    const PT ps = act ? penc[s] : (PT)0;
    KT k[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) k[c] = KINF;
    uint32_t flag = 0, mp01 = 0, mp23 = 0;
    int C = 2, lc = 1;
    if (kind == OP_R0 || kind == OP_REP) {
        PT v0 = 0, v1 = 0;
        if (act) lane_sums<T>(row, nv, kind == OP_REP, v0, v1);
        if (kind == OP_R0) {
            // Rate-0 (Sec. III-B): no fork, penalty += sum |min(a, 0)|, beta = 0.
            if (act) {
                penc[s] = ps + v0;
                for (int w = 0; w < bw; ++w) bout[s * ostride + w] = 0u;
                if (!dest) bidxc[s * 16 + j] = (uint8_t)s;
            }
            return;
        }
        // Repetition (Sec. III-E): the ML word listed first.
        flag = (v0 <= v1) ? 0u : 1u;
        k[0] = Arith<T>::mk(ps + (flag ? v1 : v0), s * 2 + 0);
        k[1] = Arith<T>::mk(ps + (flag ? v0 : v1), s * 2 + 1);
    } else {
        LK top[4];
        int neg = 0;
        if (kind == OP_R1) lane_lrb<T, 2>(row, nv, top, neg);
        else lane_lrb<T, 4>(row, nv, top, neg);
        PT ar[4];
        uint32_t m[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            ar[r] = Arith<T>::unabs((uint32_t)(top[r] >> 12));
            m[r] = (uint32_t)(top[r] & 0xFFFu);
        }
        mp01 = m[0] | (m[1] << 16);
        mp23 = m[2] | (m[3] << 16);
        if (kind == OP_R1) {
            // Rate-1 (Sec. III-C): HD, HD^m1, HD^m2, HD^m1^m2.
            C = 4;
            lc = 2;
            k[0] = Arith<T>::mk(ps, s * 4 + 0);
            k[1] = Arith<T>::mk(ps + ar[0], s * 4 + 1);
            k[2] = Arith<T>::mk(ps + ar[1], s * 4 + 2);
            k[3] = Arith<T>::mk(ps + (ar[0] + ar[1]), s * 4 + 3);
        } else {
            // SPC (Sec. III-D): ML = HD or HD^m1; ML ^ T, penalty from Eq. (9).
            C = L == 2 ? 2 : 8;
            lc = L == 2 ? 1 : 3;
            flag = (neg & 1) ? 0u : 1u;   // q
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (c < C) {
                    const uint32_t dm = spc_tmask(c) ^ (flag ? 0u : 1u);
                    PT inc = (PT)0;
                    bool first = true;
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if ((dm >> r) & 1u) { inc = first ? ar[r] : inc + ar[r]; first = false; }
                    k[c] = Arith<T>::mk(ps + inc, s * C + c);
                }
            }
            if (C == 8) sort8(k);
        }
    }
    if (!act) {
#pragma unroll
        for (int c = 0; c < 8; ++c) k[c] = KINF;
    }
    // selection (Algorithm 1); for codes that pack (L <= 16) inside an L-lane
    // segment (shorter sorting networks; the lanes past L hold no keys)
    const int nc = La * C;
    KT *tab = reinterpret_cast<KT *>(S + lay.surv);
    const bool seg = SEG && cv.pack;
    const int ls = lane & (L - 1);
    const KT tau = (nc > L) ? (seg ? warp_kth_seg(k, C, L, La, lane & ~(L - 1), ls, tab) : warp_kth(k, C, L, La, lane, tab))
                            : KINF;
    uint32_t sm = 0;
#pragma unroll
    for (int r = 0; r < 8; ++r)
        if (k[r] != KINF && k[r] <= tau) sm |= 1u << (Arith<T>::kidx(k[r]) & (uint32_t)(C - 1));
    const int base = seg ? seg_excl_scan(__popc(sm), ls, L) : warp_excl_scan(__popc(sm), lane);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        if (k[r] != KINF && k[r] <= tau) {
            const int c = (int)(Arith<T>::kidx(k[r]) & (uint32_t)(C - 1));
            tab[base + __popc(sm & ((1u << c) - 1u))] = k[r];
        }
    }
    __syncwarp();
    // commit: new slot t (lane t) takes source s's rows, the new penalty and the candidate beta
    const int La2 = nc < L ? nc : L;
    const bool act2 = lane < La2;
    const KT kt = act2 ? tab[lane] : (KT)0;
    const uint32_t ci = Arith<T>::kidx(kt);
    const int src = act2 ? (int)(ci >> lc) : 0;
    const int c = (int)(ci & (uint32_t)(C - 1));
    const uint32_t fl_s = __shfl_sync(FULL, flag, src);
    const uint32_t m01 = __shfl_sync(FULL, mp01, src);
    const uint32_t m23 = __shfl_sync(FULL, mp23, src);
    if (act2) {
        const int nxt = cur ^ 1;
        uint8_t *idxn = S + lay.idx[nxt];
        uint8_t *bidxn = S + lay.bidx[nxt];
        reinterpret_cast<PT *>(S + lay.pen[nxt])[lane] = Arith<T>::kpen(kt);
        reinterpret_cast<uint4 *>(idxn)[lane] = reinterpret_cast<const uint4 *>(idxc)[src];
        reinterpret_cast<uint4 *>(bidxn)[lane] = reinterpret_cast<const uint4 *>(bidxc)[src];
        if (!dest) bidxn[lane * 16 + j] = (uint8_t)lane;
        uint32_t *ob = bout + lane * ostride;
        if (kind == OP_REP) {
            const uint32_t word = ((fl_s != 0u) != (c == 1)) ? 0xffffffffu : 0u;
            for (int w = 0; w < bw; ++w) ob[w] = word;
        } else {
            const uint32_t dm = (kind == OP_R1) ? (uint32_t)c : (spc_tmask(c) ^ (fl_s ? 0u : 1u));
            const uint32_t mm[4] = {m01 & 0xFFFFu, m01 >> 16, m23 & 0xFFFFu, m23 >> 16};
            const T *srow = stj + (j == n ? 0 : ((int)idxc[src * 16 + j] << j));
            for (int w = 0; w < bw; ++w) {
                uint32_t word = hd_word<T>(srow + (w << 5));
#pragma unroll
                for (int rr = 0; rr < 4; ++rr)
                    if (((dm >> rr) & 1u) && (int)(mm[rr] >> 5) == w) word ^= 1u << (mm[rr] & 31u);
                ob[w] = word;
            }
        }
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Decode one frame: channel row -> payload bits, penalty, CRC flag, slot.
// Called by all W*32 threads of one frame group.
template <typename T, int W, bool SEG>
__device__ __forceinline__ void decode_frame(const CodeView &cv, uint8_t *S, uint8_t *Gs, const uint8_t *src,
                                             uint8_t *bits_row, float *pm_out, uint8_t *ok_out, int32_t *slot_out,
                                             int gidx, int gtid, bool lockstep, uint32_t sstride, uint64_t gstride,
                                             int gpc) {
    typedef typename Arith<T>::P PT;
    constexpr int GT = W * 32;
    const Layout &lay = cv.lay;
    const int lane = gtid & 31;
    const int wig = gtid >> 5;
    const int n = cv.n, N = cv.N, L = cv.L;
    // register subtrees of several frames in one warp (codes that pack: L <= 16,
    // one warp per frame; in lockstep rounds with 32 / L frame groups to a CTA).
    // Only the SEG instantiations hold that code.
    static_assert(!SEG || W == 1, "packing needs one warp per frame");
    const bool pack = SEG && cv.pack && lockstep && 32 / L <= gpc;
    const int bwn = beta_words(n);
    T *chan = chan_ptr<T>(lay, S, Gs);
    uint32_t *br = br_ptr(lay, S, Gs);
    uint32_t *ubuf = reinterpret_cast<uint32_t *>(S + lay.ubuf);

    // ---------------- channel LLRs -> stage n ----------------
    {
        const size_t nbytes = (size_t)N * sizeof(T);
        if (((reinterpret_cast<uintptr_t>(src) & 15u) == 0) && (nbytes & 15u) == 0) {
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
            uint4 *d4 = reinterpret_cast<uint4 *>(chan);
            for (int t = gtid; t < (int)(nbytes >> 4); t += GT) {
                uint4 v = __ldcs(s4 + t);
                if (sizeof(T) == 1) {   // read -128 as -127
                    v.x = __vmaxs4(v.x, 0x81818181u); v.y = __vmaxs4(v.y, 0x81818181u);
                    v.z = __vmaxs4(v.z, 0x81818181u); v.w = __vmaxs4(v.w, 0x81818181u);
                }
                d4[t] = v;
            }
        } else {
            for (int t = gtid; t < N; t += GT) {
                T v = reinterpret_cast<const T *>(src)[t];
                if (sizeof(T) == 1 && (int)v < -127) v = (T)-127;
                chan[t] = v;
            }
        }
    }
    // index tables start at row 0 so that no entry can point outside a stage
    for (int t = gtid; t < L * 4; t += GT) {
        reinterpret_cast<uint32_t *>(S + lay.idx[0])[t] = 0u;
        reinterpret_cast<uint32_t *>(S + lay.idx[1])[t] = 0u;
        reinterpret_cast<uint32_t *>(S + lay.bidx[0])[t] = 0u;
        reinterpret_cast<uint32_t *>(S + lay.bidx[1])[t] = 0u;
    }
    int La = 1, cur = 0;
    if (gtid == 0) reinterpret_cast<PT *>(S + lay.pen[0])[0] = (PT)0;
    gsync<W>(gidx);

    uint32_t op = __ldg(cv.ops);
    for (int o = 0; o < cv.n_ops; ++o) {
        uint32_t opn = (o + 1 < cv.n_ops) ? __ldg(cv.ops + o + 1) : 0u;
        const uint32_t kind = op_kind(op);
        const int j = op_stage(op);
        const int dest = op_dest(op);
        const bool solo = op_solo(op);
        const int tid = solo ? lane : gtid;
        const int nthr = solo ? 32 : GT;
        uint8_t *idxc = S + lay.idx[cur];
        uint8_t *bidxc = S + lay.bidx[cur];

        if ((kind == OP_F || kind == OP_G) && ((lay.virt_mask >> (j - 1)) & 3u)) {
            // input stage j is evaluated from the channel; an output stage that is
            // evaluated too is left to its readers
            if (!((lay.virt_mask >> (j - 1)) & 1u) && (!solo || wig == 0)) {
                const uint32_t s0 = op_start(op);
                const bool isG = kind == OP_G;
                const int D = n - j;
                if (D == 1) fg_virtual<T, 1>(lay, S, Gs, chan, idxc, bidxc, isG, j, s0, La, tid, nthr);
                else if (D == 2) fg_virtual<T, 2>(lay, S, Gs, chan, idxc, bidxc, isG, j, s0, La, tid, nthr);
                else fg_virtual<T, 3>(lay, S, Gs, chan, idxc, bidxc, isG, j, s0, La, tid, nthr);
            }
        } else if ((sizeof(T) == 1 || (SEG && L <= 8)) && (kind == OP_F || kind == OP_G) && op_kind(opn) == OP_F &&
                   op_stage(opn) == j - 1 && j - 2 >= 5 && ((lay.virt_mask >> (j - 2)) & 7u) == 0) {
            // ------------ F or G, then the child's F: stage j -> j-1 -> j-2 ------------
            // The child that stage j-1 feeds (the left one after F, the right
            // one after G) is an inner node too, so its F comes next. Each item
            // reads the four quarter rows of stage j at one offset (and, for G,
            // the left child's beta bits there), writes both halves of stage
            // j-1 (the child's G reads them later) and, from the same
            // registers, stage j-2: one pass and one dependent round trip fewer
            // than two operations. Measured faster for int8 at every L and for
            // float at L <= 8, slower for float at L = 16 / 32 (four items in
            // flight per thread instead of eight). Float takes it only in the
            // packed instantiations (L <= 4 by default): compiled into the
            // kernel that L = 32 runs, the unused code alone cost it about 1 %.
            if (!solo || wig == 0) {
                const int q = 1 << (j - 2);
                const bool isG = kind == OP_G;
                const T *inb = (j == n) ? chan : alpha_ptr<T>(lay, S, Gs, j);
                T *o1b = alpha_ptr<T>(lay, S, Gs, j - 1);
                T *o2b = alpha_ptr<T>(lay, S, Gs, j - 2);
                const uint32_t *blb = bl_ptr(lay, S, Gs, j - 1);
                const int bwc = beta_words(j - 1);
                if (sizeof(T) == 4) {
                    const int lv = j - 4;              // float4 items per quarter row (q >= 32)
                    const int total = La << lv;
                    for (int t0 = tid; t0 < total; t0 += 4 * nthr) {
                        float4 a[4][4];
                        uint32_t nb0[4] = {0u, 0u, 0u, 0u}, nb1[4] = {0u, 0u, 0u, 0u};
                        int pp[4], vv[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int t = t0 + u * nthr;
                            pp[u] = t < total ? t >> lv : 0;
                            vv[u] = t < total ? t & ((1 << lv) - 1) : 0;
                            const float4 *in = reinterpret_cast<const float4 *>(
                                reinterpret_cast<const float *>(inb) + (j == n ? 0 : ((int)idxc[pp[u] * 16 + j] << j)));
#pragma unroll
                            for (int r = 0; r < 4; ++r) a[u][r] = in[vv[u] + r * (q >> 2)];
                            if (isG) {
                                const uint32_t *bl = blb + (int)bidxc[pp[u] * 16 + j - 1] * bwc;
                                const int i0 = vv[u] << 2, i1 = i0 + q;
                                nb0[u] = bl[i0 >> 5] >> (i0 & 31);
                                nb1[u] = bl[i1 >> 5] >> (i1 & 31);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            if (t0 + u * nthr >= total) break;
                            float4 e0, e1, r;
                            if (isG) {
                                e0.x = g_op(a[u][0].x, a[u][2].x, nb0[u] & 1u);
                                e0.y = g_op(a[u][0].y, a[u][2].y, (nb0[u] >> 1) & 1u);
                                e0.z = g_op(a[u][0].z, a[u][2].z, (nb0[u] >> 2) & 1u);
                                e0.w = g_op(a[u][0].w, a[u][2].w, (nb0[u] >> 3) & 1u);
                                e1.x = g_op(a[u][1].x, a[u][3].x, nb1[u] & 1u);
                                e1.y = g_op(a[u][1].y, a[u][3].y, (nb1[u] >> 1) & 1u);
                                e1.z = g_op(a[u][1].z, a[u][3].z, (nb1[u] >> 2) & 1u);
                                e1.w = g_op(a[u][1].w, a[u][3].w, (nb1[u] >> 3) & 1u);
                            } else {
                                e0.x = f_op(a[u][0].x, a[u][2].x); e0.y = f_op(a[u][0].y, a[u][2].y);
                                e0.z = f_op(a[u][0].z, a[u][2].z); e0.w = f_op(a[u][0].w, a[u][2].w);
                                e1.x = f_op(a[u][1].x, a[u][3].x); e1.y = f_op(a[u][1].y, a[u][3].y);
                                e1.z = f_op(a[u][1].z, a[u][3].z); e1.w = f_op(a[u][1].w, a[u][3].w);
                            }
                            r.x = f_op(e0.x, e1.x); r.y = f_op(e0.y, e1.y); r.z = f_op(e0.z, e1.z); r.w = f_op(e0.w, e1.w);
                            float4 *o1 = reinterpret_cast<float4 *>(reinterpret_cast<float *>(o1b) + (pp[u] << (j - 1)));
                            o1[vv[u]] = e0;
                            o1[vv[u] + (q >> 2)] = e1;
                            reinterpret_cast<float4 *>(reinterpret_cast<float *>(o2b) + (pp[u] << (j - 2)))[vv[u]] = r;
                        }
                    }
                } else {
                    const int lv = j - 6;              // 16-byte items per quarter row (q >= 32)
                    const int total = La << lv;
                    for (int t0 = tid; t0 < total; t0 += 2 * nthr) {
                        uint4 a[2][4];
                        uint32_t nb0[2] = {0u, 0u}, nb1[2] = {0u, 0u};
                        int pp[2], vv[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int t = t0 + u * nthr;
                            pp[u] = t < total ? t >> lv : 0;
                            vv[u] = t < total ? t & ((1 << lv) - 1) : 0;
                            const uint4 *in = reinterpret_cast<const uint4 *>(
                                reinterpret_cast<const int8_t *>(inb) + (j == n ? 0 : ((int)idxc[pp[u] * 16 + j] << j)));
#pragma unroll
                            for (int r = 0; r < 4; ++r) a[u][r] = in[vv[u] + r * (q >> 4)];
                            if (isG) {
                                const uint32_t *bl = blb + (int)bidxc[pp[u] * 16 + j - 1] * bwc;
                                const int i0 = vv[u] << 4, i1 = i0 + q;
                                nb0[u] = bl[i0 >> 5] >> (i0 & 31);
                                nb1[u] = bl[i1 >> 5] >> (i1 & 31);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            if (t0 + u * nthr >= total) break;
                            uint4 e0, e1, r;
                            if (isG) {
                                e0.x = g4(a[u][0].x, a[u][2].x, nb0[u] & 15u);
                                e0.y = g4(a[u][0].y, a[u][2].y, (nb0[u] >> 4) & 15u);
                                e0.z = g4(a[u][0].z, a[u][2].z, (nb0[u] >> 8) & 15u);
                                e0.w = g4(a[u][0].w, a[u][2].w, (nb0[u] >> 12) & 15u);
                                e1.x = g4(a[u][1].x, a[u][3].x, nb1[u] & 15u);
                                e1.y = g4(a[u][1].y, a[u][3].y, (nb1[u] >> 4) & 15u);
                                e1.z = g4(a[u][1].z, a[u][3].z, (nb1[u] >> 8) & 15u);
                                e1.w = g4(a[u][1].w, a[u][3].w, (nb1[u] >> 12) & 15u);
                            } else {
                                e0.x = f4(a[u][0].x, a[u][2].x); e0.y = f4(a[u][0].y, a[u][2].y);
                                e0.z = f4(a[u][0].z, a[u][2].z); e0.w = f4(a[u][0].w, a[u][2].w);
                                e1.x = f4(a[u][1].x, a[u][3].x); e1.y = f4(a[u][1].y, a[u][3].y);
                                e1.z = f4(a[u][1].z, a[u][3].z); e1.w = f4(a[u][1].w, a[u][3].w);
                            }
                            r.x = f4(e0.x, e1.x); r.y = f4(e0.y, e1.y); r.z = f4(e0.z, e1.z); r.w = f4(e0.w, e1.w);
                            uint4 *o1 = reinterpret_cast<uint4 *>(reinterpret_cast<int8_t *>(o1b) + (pp[u] << (j - 1)));
                            o1[vv[u]] = e0;
                            o1[vv[u] + (q >> 4)] = e1;
                            reinterpret_cast<uint4 *>(reinterpret_cast<int8_t *>(o2b) + (pp[u] << (j - 2)))[vv[u]] = r;
                        }
                    }
                }
                for (int t = tid; t < La; t += nthr) {
                    idxc[t * 16 + j - 1] = (uint8_t)t;
                    idxc[t * 16 + j - 2] = (uint8_t)t;
                }
            }
            // the child's F is done: its flags (sync) close this operation
            ++o;
            op = opn;
            opn = (o + 1 < cv.n_ops) ? __ldg(cv.ops + o + 1) : 0u;
        } else if (kind == OP_F || kind == OP_G) {
            if (!solo || wig == 0) {
                // ---------------- F / G: stage j -> stage j-1 ----------------
                const int jo = j - 1;
                const int h = 1 << jo;
                const T *inb = (j == n) ? chan : alpha_ptr<T>(lay, S, Gs, j);
                T *outb = alpha_ptr<T>(lay, S, Gs, jo);
                const bool isG = kind == OP_G;
                const uint32_t *blb = bl_ptr(lay, S, Gs, jo);
                const int bwc = beta_words(jo);
                if (sizeof(T) == 4) {
                    const int lv = jo - 2;             // h >= 16 here: float4 items, eight in flight per thread
                    const int total = La << lv;
                    for (int t0 = tid; t0 < total; t0 += 8 * nthr) {
                        float4 a[8], b[8];
                        uint32_t nb[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
                        int pp[8], vv[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int t = t0 + u * nthr;
                            pp[u] = t < total ? t >> lv : 0;
                            vv[u] = t < total ? t & ((1 << lv) - 1) : 0;
                            const float *in = reinterpret_cast<const float *>(inb) +
                                              (j == n ? 0 : ((int)idxc[pp[u] * 16 + j] << j));
                            a[u] = reinterpret_cast<const float4 *>(in)[vv[u]];
                            b[u] = reinterpret_cast<const float4 *>(in + h)[vv[u]];
                            if (isG) {
                                const int i = vv[u] << 2;
                                nb[u] = blb[(int)bidxc[pp[u] * 16 + jo] * bwc + (i >> 5)] >> (i & 31);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            if (t0 + u * nthr >= total) break;
                            float4 r;
                            if (isG) {
                                r.x = g_op(a[u].x, b[u].x, nb[u] & 1u); r.y = g_op(a[u].y, b[u].y, (nb[u] >> 1) & 1u);
                                r.z = g_op(a[u].z, b[u].z, (nb[u] >> 2) & 1u); r.w = g_op(a[u].w, b[u].w, (nb[u] >> 3) & 1u);
                            } else {
                                r.x = f_op(a[u].x, b[u].x); r.y = f_op(a[u].y, b[u].y);
                                r.z = f_op(a[u].z, b[u].z); r.w = f_op(a[u].w, b[u].w);
                            }
                            reinterpret_cast<float4 *>(reinterpret_cast<float *>(outb) + (pp[u] << jo))[vv[u]] = r;
                        }
                    }
                } else {
                    const int lv = jo - 4;             // h >= 16 here: 16-byte items
                    const int total = La << lv;
                    for (int t0 = tid; t0 < total; t0 += 2 * nthr) {
                        uint4 a[2], b[2];
                        uint32_t nb[2] = {0u, 0u};
                        int pp[2], vv[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const int t = t0 + u * nthr;
                            pp[u] = t < total ? t >> lv : 0;
                            vv[u] = t < total ? t & ((1 << lv) - 1) : 0;
                            const int8_t *in = reinterpret_cast<const int8_t *>(inb) +
                                               (j == n ? 0 : ((int)idxc[pp[u] * 16 + j] << j));
                            a[u] = reinterpret_cast<const uint4 *>(in)[vv[u]];
                            b[u] = reinterpret_cast<const uint4 *>(in + h)[vv[u]];
                            if (isG) {
                                const int i = vv[u] << 4;
                                nb[u] = blb[(int)bidxc[pp[u] * 16 + jo] * bwc + (i >> 5)] >> (i & 31);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            if (t0 + u * nthr >= total) break;
                            uint4 r;
                            if (isG) {
                                r.x = g4(a[u].x, b[u].x, nb[u] & 15u); r.y = g4(a[u].y, b[u].y, (nb[u] >> 4) & 15u);
                                r.z = g4(a[u].z, b[u].z, (nb[u] >> 8) & 15u); r.w = g4(a[u].w, b[u].w, (nb[u] >> 12) & 15u);
                            } else {
                                r.x = f4(a[u].x, b[u].x); r.y = f4(a[u].y, b[u].y);
                                r.z = f4(a[u].z, b[u].z); r.w = f4(a[u].w, b[u].w);
                            }
                            reinterpret_cast<uint4 *>(reinterpret_cast<int8_t *>(outb) + (pp[u] << jo))[vv[u]] = r;
                        }
                    }
                }
                for (int t = tid; t < La; t += nthr) idxc[t * 16 + jo] = (uint8_t)t;
            }
        } else if (kind == OP_COMB) {
            if (!solo || wig == 0) {
                // ---------------- Combine: [beta_l ^ beta_r, beta_r] ----------------
                const int jc = j - 1;                  // >= kSubLog
                const int bwc = beta_words(jc);
                const uint32_t *blb = bl_ptr(lay, S, Gs, jc);
                uint32_t *out = dest ? br : bl_ptr(lay, S, Gs, j);
                const int ostride = dest ? bwn : beta_words(j);
                if (jc >= 5) {
                    const int lw = jc - 5;
                    const int total = La << lw;
                    for (int t = tid; t < total; t += nthr) {
                        const int p = t >> lw, w = t & (bwc - 1);
                        const uint32_t l = blb[(int)bidxc[p * 16 + jc] * bwc + w];
                        const uint32_t r = br[p * bwn + w];
                        uint32_t *o2 = out + p * ostride;
                        o2[w] = l ^ r;
                        o2[w + bwc] = r;
                    }
                } else {
                    const int h = 1 << jc;
                    const uint32_t m = (1u << h) - 1u;
                    for (int t = tid; t < La; t += nthr) {
                        const uint32_t l = blb[(int)bidxc[t * 16 + jc]];
                        const uint32_t r = br[t * bwn];
                        out[t * ostride] = ((l ^ r) & m) | ((r & m) << h);
                    }
                }
                if (!dest)
                    for (int t = tid; t < La; t += nthr) bidxc[t * 16 + j] = (uint8_t)t;
            }
        } else if (kind == OP_SUB) {
            // ---------------- a small subtree in registers (warp 0) ----------------
            if (pack) {
                // L <= 16 in lockstep: the first warp of every run of P = 32 / L
                // groups runs the subtree for all P frames, L lanes each, and
                // the others wait at the CTA barrier below
                if ((gidx & (32 / L - 1)) == 0) {
                    const int P = 32 / L;
                    if (j == kSubLog) run_sub<T, 4, true>(cv, S, Gs, op, La, cur, lane, P, sstride, gstride);
                    else if (j == kSubLog + 1) run_sub32<T, true>(cv, S, Gs, op, La, cur, lane, P, sstride, gstride);
                    else run_sub<T, 3, true>(cv, S, Gs, op, La, cur, lane, P, sstride, gstride);
                }
                asm volatile("bar.sync 15, %0;" ::"r"(blockDim.x) : "memory");
            } else if (SEG && cv.pack && wig == 0) {
                // one frame, its selection in an L-lane segment (shorter sorting
                // networks); the other lanes idle
                if (j == kSubLog) run_sub<T, 4, true>(cv, S, Gs, op, La, cur, lane);
                else if (j == kSubLog + 1) run_sub32<T, true>(cv, S, Gs, op, La, cur, lane);
                else run_sub<T, 3, true>(cv, S, Gs, op, La, cur, lane);
            } else if (wig == 0) {
                if (j == kSubLog) run_sub<T, 4, false>(cv, S, Gs, op, La, cur, lane);
                else if (j == kSubLog + 1) run_sub32<T, false>(cv, S, Gs, op, La, cur, lane);
                else run_sub<T, 3, false>(cv, S, Gs, op, La, cur, lane);
            }
            const int lm = op_sub_logmult(op);
            La = (lm >= 6 || (La << lm) > L) ? L : (La << lm);
            if (op_sub_fork(op)) cur ^= 1;
        } else {
            // ---------------- a leaf of more than 16 bits (warp 0) ----------------
            if (wig == 0) big_leaf<T, SEG>(cv, S, Gs, kind, j, dest, La, cur, lane);
            if (kind != OP_R0) {
                const int C = kind == OP_R1 ? 4 : (kind == OP_REP ? 2 : (L == 2 ? 2 : 8));
                La = La * C < L ? La * C : L;
                cur ^= 1;
            }
        }
        if (op_sync(op)) gsync<W>(gidx);
        else if (wig == 0) __syncwarp();
        // Every group of the CTA runs the same schedule: a CTA barrier before
        // each register subtree (the largest code) keeps them on the same
        // instructions there, so they share instruction fetches; between the
        // barriers the other ops may drift and overlap their latencies.
        if (lockstep && op_kind(opn) == OP_SUB) asm volatile("bar.sync 15, %0;" ::"r"(blockDim.x) : "memory");
        op = opn;
    }
    gsync<W>(gidx);

    // ---------------- final pick (Sec. II-B) ----------------
    PT *penc = reinterpret_cast<PT *>(S + lay.pen[cur]);
    uint32_t *synb = reinterpret_cast<uint32_t *>(S + lay.surv);
    if (cv.crc_len > 0) {
        const int nbytes = N >> 3;
        for (int p = wig; p < La; p += W) {
            const uint8_t *xb = reinterpret_cast<const uint8_t *>(br + p * bwn);
            uint32_t acc = 0;
            for (int b = lane; b < nbytes; b += 32) acc ^= __ldg(cv.syn + ((b << 8) | xb[b]));
            for (int off = 16; off >= 1; off >>= 1) acc ^= __shfl_xor_sync(FULL, acc, off);
            if (lane == 0) synb[p] = acc;
        }
    }
    gsync<W>(gidx);
    if (wig == 0) {
        unsigned long long key = ~0ull;
        if (lane < La) {
            const bool okp = cv.crc_len == 0 || synb[lane] == 0u;
            key = ((unsigned long long)(okp ? 0u : 1u) << 63) |
                  ((unsigned long long)Arith<T>::pbits(penc[lane]) << 8) | (unsigned long long)lane;
        }
        for (int off = 16; off >= 1; off >>= 1) {
            const unsigned long long o2 = __shfl_xor_sync(FULL, key, off);
            key = o2 < key ? o2 : key;
        }
        const int win = (int)(key & 0xFFu);
        const uint32_t okw = (uint32_t)(key >> 63) ^ 1u;
        // u = x G_N for the winner (natural-order butterflies); a systematic
        // code keeps x, whose information positions carry payload and CRC
        const uint32_t *xw = br + win * bwn;
        const int R = bwn > 32 ? bwn >> 5 : 1;
        uint32_t U[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int w = lane + 32 * r;
            U[r] = (r < R && w < bwn) ? xw[w] : 0u;
        }
        if (!cv.systematic) {
            const uint32_t M[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
#pragma unroll
                for (int e = 0; e < 5; ++e) {
                    const int hb = 1 << e;
                    if (hb < N) U[r] ^= (U[r] >> hb) & M[e];
                }
            }
            for (int d = 1; d < bwn; d <<= 1) {
                if (d >= 32) {
                    const int dr = d >> 5;
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        if (r < R && !(r & dr) && r + dr < 4) U[r] ^= U[r + dr];
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const uint32_t v = __shfl_down_sync(FULL, U[r], d);
                        if (!(lane & d)) U[r] ^= v;
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int w = lane + 32 * r;
            if (r < R && w < bwn) ubuf[w] = U[r];
        }
        if (lane == 0) {
            *pm_out = Arith<T>::to_out(penc[win]);
            if (ok_out) *ok_out = (uint8_t)okw;
            if (slot_out) *slot_out = win;
        }
    }
    gsync<W>(gidx);
    for (int b = gtid; b < cv.kb; b += GT) {
        uint32_t byte = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int pos = 8 * b + t;
            if (pos < cv.k) {
                const uint32_t u = __ldg(cv.info + pos);
                byte |= ((ubuf[u >> 5] >> (u & 31u)) & 1u) << t;
            }
        }
        bits_row[b] = (uint8_t)byte;
    }
    gsync<W>(gidx);
}

// Plain form: one code, frames f = group, group + n_groups, ...
template <typename T, int W, bool SEG>
__global__ void __launch_bounds__(kMaxCtaThreads) decode_kernel(const Params P) {
    constexpr int GT = W * 32;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int gidx = threadIdx.x / GT;
    const int gtid = threadIdx.x - gidx * GT;
    uint8_t *S = smem_raw + (size_t)gidx * P.cv.lay.bytes;
    const int ggid = blockIdx.x * P.groups_per_cta + gidx;
    const int ngroups = gridDim.x * P.groups_per_cta;
    uint8_t *Gs = P.scratch ? P.scratch + (size_t)ggid * P.cv.lay.gbytes : nullptr;
    const size_t nbytes = (size_t)P.cv.N * sizeof(T);
    const uint32_t nf = P.frame_idx ? *P.frame_cnt : P.n_frames;
    for (uint32_t i = ggid; i < nf; i += ngroups) {
        const uint32_t f = P.frame_idx ? P.frame_idx[i] : i;
        // lockstep only in rounds where every group of the CTA has a frame, so
        // that all warps reach each per-op barrier the same number of times
        const bool full = P.groups_per_cta > 1 && (i - (uint32_t)gidx) + (uint32_t)P.groups_per_cta <= nf;
        decode_frame<T, W, SEG>(P.cv, S, Gs, reinterpret_cast<const uint8_t *>(P.llr) + (size_t)f * nbytes,
                           P.bits + (size_t)f * P.cv.kb, P.pm + f, P.ok ? P.ok + f : nullptr,
                           P.slot ? P.slot + f : nullptr, gidx, gtid, full, P.cv.lay.bytes, P.cv.lay.gbytes,
                           P.groups_per_cta);
    }
}

// Compaction for the adaptive decoder (Sec. V): indices of frames whose CRC
// failed. One warp-aggregated atomic per warp; the order is unspecified.
__global__ void crc_failures_kernel(const uint8_t *ok, uint32_t n, uint32_t *idx, uint32_t *cnt) {
    const uint32_t lane = threadIdx.x & 31u;
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n;
         base += gridDim.x * blockDim.x) {
        const uint32_t f = base + lane;
        const bool bad = f < n && ok[f] == 0;
        const uint32_t m = __ballot_sync(FULL, bad);
        if (!m) continue;
        uint32_t off = 0;
        if (lane == 0) off = atomicAdd(cnt, (uint32_t)__popc(m));
        off = __shfl_sync(FULL, off, 0);
        if (bad) idx[off + __popc(m & ((1u << lane) - 1u))] = f;
    }
}

// Batched form: frames of several codes in one persistent launch. A CTA takes
// one work item per group (items ordered by decreasing cost, each class's
// items contiguous) from a device counter; the code of an item is copied into
// the group's shared memory when it changes. When all groups of the CTA got a
// frame of the same code they run it in lockstep, as in the plain form.
template <typename T, int W, bool SEG>
__global__ void __launch_bounds__(kMaxCtaThreads) batch_kernel(const BatchParams B) {
    constexpr int GT = W * 32;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int gidx = threadIdx.x / GT;
    const int gtid = threadIdx.x - gidx * GT;
    uint8_t *region = smem_raw + (size_t)gidx * B.group_bytes;
    CodeView *cvs = reinterpret_cast<CodeView *>(region);
    uint32_t *slot_word = reinterpret_cast<uint32_t *>(region + sizeof(CodeView));
    uint8_t *S = region + B.view_bytes;
    const int ggid = blockIdx.x * B.groups_per_cta + gidx;
    uint8_t *Gs = B.scratch ? B.scratch + (size_t)ggid * B.gbytes : nullptr;
    // the CTA's work slot is group 0's
    uint32_t *cta_slot = reinterpret_cast<uint32_t *>(smem_raw + sizeof(CodeView));
    uint32_t loaded = 0xffffffffu;
    (void)slot_word;
    for (;;) {
        if (threadIdx.x == 0) *cta_slot = atomicAdd(B.counter, (uint32_t)B.groups_per_cta);
        __syncthreads();
        const uint32_t base = *cta_slot;
        const uint32_t it = base + (uint32_t)gidx;
        const bool have = it < B.n_items;
        const uint32_t cls = have ? B.items[it].cls : 0xffffffffu;
        const uint32_t cls0 = base < B.n_items ? B.items[base].cls : 0xfffffffeu;
        // also orders the read of the slot above before its next write
        const bool lock = __syncthreads_and(have && cls == cls0) && B.groups_per_cta > 1;
        if (base >= B.n_items) break;
        if (!have) continue;
        const BatchItem item = B.items[it];
        if (item.cls != loaded) {
            const uint32_t *srcw = reinterpret_cast<const uint32_t *>(B.classes + item.cls);
            uint32_t *dstw = reinterpret_cast<uint32_t *>(cvs);
            for (int t = gtid; t < (int)(sizeof(CodeView) / 4); t += GT) dstw[t] = srcw[t];
            loaded = item.cls;
            gsync<W>(gidx);
        }
        decode_frame<T, W, SEG>(*cvs, S, Gs, B.llr + item.llr_off, B.bits + item.bits_off, B.pm + item.frame,
                           B.ok ? B.ok + item.frame : nullptr, B.slot ? B.slot + item.frame : nullptr, gidx, gtid,
                           lock, B.group_bytes, B.gbytes, B.groups_per_cta);
    }
}

template <typename T, int W, bool SEG = false>
cudaError_t launch_one(const LaunchShape &sh, const Params &p, int grid, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(decode_kernel<T, W, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sh.smem);
    if (e != cudaSuccess) return e;
    decode_kernel<T, W, SEG><<<grid, sh.threads, sh.smem, st>>>(p);
    return cudaGetLastError();
}

template <typename T, int W, bool SEG = false>
int occ_one(const LaunchShape &sh) {
    if (cudaFuncSetAttribute(decode_kernel<T, W, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, decode_kernel<T, W, SEG>, sh.threads, sh.smem) !=
        cudaSuccess)
        return 0;
    return nb;
}

template <typename T, int W, bool SEG = false>
cudaError_t launch_batch_one(const BatchParams &b, int grid, uint32_t smem, int threads, cudaStream_t st) {
    cudaError_t e =
        cudaFuncSetAttribute(batch_kernel<T, W, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    batch_kernel<T, W, SEG><<<grid, threads, smem, st>>>(b);
    return cudaGetLastError();
}

template <typename T, int W, bool SEG = false>
int occ_batch_one(uint32_t smem, int threads) {
    if (cudaFuncSetAttribute(batch_kernel<T, W, SEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<T, W, SEG>, threads, smem) != cudaSuccess)
        return 0;
    return nb;
}

// One type's kernels behind one entry each (shape -> instantiation).
template <typename T>
cudaError_t launch_decode_typed(const LaunchShape &sh, const Params &p, int grid, cudaStream_t st) {
    if (sh.pack && sh.warps == 1) return launch_one<T, 1, true>(sh, p, grid, st);
    if (sh.warps == 1) return launch_one<T, 1>(sh, p, grid, st);
    if (sh.warps == 2) return launch_one<T, 2>(sh, p, grid, st);
    if (sh.warps == 4) return launch_one<T, 4>(sh, p, grid, st);
    return cudaErrorInvalidValue;
}

template <typename T>
int occupancy_typed(const LaunchShape &sh) {
    if (sh.pack && sh.warps == 1) return occ_one<T, 1, true>(sh);
    if (sh.warps == 1) return occ_one<T, 1>(sh);
    if (sh.warps == 2) return occ_one<T, 2>(sh);
    if (sh.warps == 4) return occ_one<T, 4>(sh);
    return 0;
}

template <typename T>
cudaError_t launch_batch_typed(int warps, bool seg, const BatchParams &b, int grid, uint32_t smem, int threads,
                               cudaStream_t st) {
    if (seg && warps == 1) return launch_batch_one<T, 1, true>(b, grid, smem, threads, st);
    if (warps == 1) return launch_batch_one<T, 1>(b, grid, smem, threads, st);
    if (warps == 2) return launch_batch_one<T, 2>(b, grid, smem, threads, st);
    if (warps == 4) return launch_batch_one<T, 4>(b, grid, smem, threads, st);
    return cudaErrorInvalidValue;
}

template <typename T>
int occupancy_batch_typed(int warps, bool seg, uint32_t smem, int threads) {
    if (seg && warps == 1) return occ_batch_one<T, 1, true>(smem, threads);
    if (warps == 1) return occ_batch_one<T, 1>(smem, threads);
    if (warps == 2) return occ_batch_one<T, 2>(smem, threads);
    if (warps == 4) return occ_batch_one<T, 4>(smem, threads);
    return 0;
}

}  // namespace

// The kernels compile in four parts, one translation unit each, so that they
// build in parallel: 0 float and 1 int8 in the plain form, 2 float and 3 int8
// in the batched form. POLAR_KPART picks one part (all four when it is not
// defined); the dispatchers sit in part 0.
#ifndef POLAR_KPART
#define POLAR_KPART -1
#endif
#define POLAR_HAS_PART(p) (POLAR_KPART < 0 || POLAR_KPART == (p))

cudaError_t launch_decode_f32(const LaunchShape &sh, const Params &p, int grid, cudaStream_t st);
cudaError_t launch_decode_i8(const LaunchShape &sh, const Params &p, int grid, cudaStream_t st);
int occupancy_f32(const LaunchShape &sh);
int occupancy_i8(const LaunchShape &sh);
cudaError_t launch_batch_f32(int warps, bool seg, const BatchParams &b, int grid, uint32_t smem, int threads,
                             cudaStream_t st);
cudaError_t launch_batch_i8(int warps, bool seg, const BatchParams &b, int grid, uint32_t smem, int threads,
                            cudaStream_t st);
int occupancy_batch_f32(int warps, bool seg, uint32_t smem, int threads);
int occupancy_batch_i8(int warps, bool seg, uint32_t smem, int threads);

#if POLAR_HAS_PART(0)
cudaError_t launch_decode_f32(const LaunchShape &sh, const Params &p, int grid, cudaStream_t st) {
    return launch_decode_typed<float>(sh, p, grid, st);
}
int occupancy_f32(const LaunchShape &sh) { return occupancy_typed<float>(sh); }
#endif
#if POLAR_HAS_PART(1)
cudaError_t launch_decode_i8(const LaunchShape &sh, const Params &p, int grid, cudaStream_t st) {
    return launch_decode_typed<int8_t>(sh, p, grid, st);
}
int occupancy_i8(const LaunchShape &sh) { return occupancy_typed<int8_t>(sh); }
#endif
#if POLAR_HAS_PART(2)
cudaError_t launch_batch_f32(int warps, bool seg, const BatchParams &b, int grid, uint32_t smem, int threads,
                             cudaStream_t st) {
    return launch_batch_typed<float>(warps, seg, b, grid, smem, threads, st);
}
int occupancy_batch_f32(int warps, bool seg, uint32_t smem, int threads) {
    return occupancy_batch_typed<float>(warps, seg, smem, threads);
}
#endif
#if POLAR_HAS_PART(3)
cudaError_t launch_batch_i8(int warps, bool seg, const BatchParams &b, int grid, uint32_t smem, int threads,
                            cudaStream_t st) {
    return launch_batch_typed<int8_t>(warps, seg, b, grid, smem, threads, st);
}
int occupancy_batch_i8(int warps, bool seg, uint32_t smem, int threads) {
    return occupancy_batch_typed<int8_t>(warps, seg, smem, threads);
}
#endif

#if POLAR_HAS_PART(0)
cudaError_t launch_crc_failures(const uint8_t *ok, uint32_t n, uint32_t *idx, uint32_t *cnt, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess || n == 0) return e;
    const int blocks = (int)std::min<uint32_t>((n + 255) / 256, 4096u);
    crc_failures_kernel<<<blocks, 256, 0, st>>>(ok, n, idx, cnt);
    return cudaGetLastError();
}

cudaError_t launch_batch(int dtype, int warps, bool seg, const BatchParams &b, int grid, uint32_t smem, int threads,
                         cudaStream_t st) {
    return dtype == 0 ? launch_batch_f32(warps, seg, b, grid, smem, threads, st)
                      : launch_batch_i8(warps, seg, b, grid, smem, threads, st);
}

int occupancy_batch(int dtype, int warps, bool seg, uint32_t smem, int threads) {
    return dtype == 0 ? occupancy_batch_f32(warps, seg, smem, threads) : occupancy_batch_i8(warps, seg, smem, threads);
}

cudaError_t launch_decode(int dtype, const LaunchShape &sh, const Params &p, int grid, cudaStream_t st) {
    return dtype == 0 ? launch_decode_f32(sh, p, grid, st) : launch_decode_i8(sh, p, grid, st);
}

int occupancy(int dtype, const LaunchShape &sh) { return dtype == 0 ? occupancy_f32(sh) : occupancy_i8(sh); }
#endif

}  // namespace polar
