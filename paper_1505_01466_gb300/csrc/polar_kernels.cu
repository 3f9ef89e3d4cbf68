// polar_kernels.cu -- list-CRC decoding of polar codes over the unrolled
// Fast-SSC tree, for GB300 (sm_103a).
//
// One frame is decoded by a group of W warps; a CTA holds 4 / W groups and
// every group loops over frames (persistent). All L paths of a frame advance
// through the same unrolled schedule in lockstep, so:
//
//  * alpha stage j holds one row of 2^j LLRs per physical slot. F and G
//    (Eq. (1), (2)) read stage j+1 through the path's index-table entry and
//    always write the path's own row of stage j: at that moment stage j is
//    dead for every path. A fork only copies the parent's 16-byte index row
//    -- the lazy copy of Sec. IV-A -- never LLRs.
//  * beta is bit-packed. Left-child outputs (BL[j]) sit behind a second
//    index table (Sec. IV-B); the right-child / root output (BR) is consumed
//    by the Combine (Eq. (3)) that follows at once and needs none.
//  * nodes of at most 16 bits are "solo": warp 0 runs them alone, one lane
//    per path for leaves, with only warp-level syncs between consecutive solo
//    operations; larger nodes use the whole group, one element per thread.
//  * a forking leaf (Sec. III-C..E) produces keys (penalty, source * C +
//    candidate) for each source path. Warp 0 keeps the L smallest
//    (Algorithm 1) without shared-memory sorting: lane s holds source s's
//    candidates sorted, the ML column is bitonic-sorted across lanes and the
//    later columns are merged in until the L-th key can no longer move.
//    Survivors take slots in (source, candidate) order by a warp prefix scan
//    and inherit their parent's index rows, penalty and candidate beta.
//  * the final pick (Sec. II-B) checks each path's CRC with byte tables of
//    the syndrome of every codeword bit, and writes the winner's payload.
//
// Float sums of many terms (Rate-0, repetition) use the pairwise tree
// s[i] = x[i] + x[i + n/2]; sums of least-reliable-bit terms run left to
// right in rank order; every new penalty is parent + increment. int8 LLRs
// use saturated G and exact integer penalties.

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
__device__ __forceinline__ int8_t f_op(int8_t a, int8_t b) {
    int x = a, y = b;
    int m = min(abs(x), abs(y));
    return (int8_t)(((x ^ y) < 0) ? -m : m);
}
__device__ __forceinline__ int8_t g_op(int8_t a, int8_t b, uint32_t beta) {
    int r = beta ? (int)b - (int)a : (int)b + (int)a;
    return (int8_t)max(-127, min(127, r));
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

template <typename T>
__device__ __forceinline__ T *stage_ptr(const Layout &lay, uint8_t *S, uint8_t *Gs, int j) {
    return ((lay.spill_mask >> j) & 1u) ? reinterpret_cast<T *>(Gs + lay.galpha[j])
                                        : reinterpret_cast<T *>(S + lay.alpha[j]);
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

// The L-th smallest key of the warp, lane s holding its keys sorted in k[].
// Column r (every lane's r-th key) can change the result only while its
// minimum is below the current L-th key; each lane's columns only grow.
template <typename K>
__device__ __forceinline__ K warp_kth(const K (&k)[8], int C, int L, int lane) {
    K B = bsort32(k[0], lane);
    K tau = __shfl_sync(FULL, B, L - 1);
#pragma unroll
    for (int r = 1; r < 8; ++r) {
        if (r >= C) break;
        K col = k[r];
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

__device__ __forceinline__ int warp_excl_scan(int v, int lane) {
    int x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(FULL, x, d);
        if (lane >= d) x += o;
    }
    return x - v;
}

// ---- canonical team sums and least reliable bits (large leaves) -----------
template <typename T>
__device__ __forceinline__ void team_sums(T *row, int K, int TS, int tl, bool act, bool want1,
                                          typename Arith<T>::P &v0, typename Arith<T>::P &v1) {
    typedef typename Arith<T>::P P;
    P s0 = 0, s1 = 0;
    if (act) {
        if (K == 1) {
            P a = Arith<T>::val(row[tl]);
            s0 = Arith<T>::negpart(a);
            s1 = Arith<T>::pospart(a);
        } else if (sizeof(T) == 4) {
            // in-lane levels of the tree, in place on the (dead) leaf input
            float *x = reinterpret_cast<float *>(row) + tl;
            const int hK = K >> 1;
            for (int k = 0; k < hK; ++k) {
                float a = x[k * TS], b = x[(k + hK) * TS];
                x[k * TS] = Arith<float>::negpart(a) + Arith<float>::negpart(b);
                if (want1) x[(k + hK) * TS] = Arith<float>::pospart(a) + Arith<float>::pospart(b);
            }
            for (int hh = hK >> 1; hh >= 1; hh >>= 1) {
                for (int k = 0; k < hh; ++k) {
                    x[k * TS] = x[k * TS] + x[(k + hh) * TS];
                    if (want1) x[(hK + k) * TS] = x[(hK + k) * TS] + x[(hK + k + hh) * TS];
                }
            }
            s0 = (P)x[0];
            s1 = want1 ? (P)x[hK * TS] : (P)0;
        } else {
            for (int k = 0; k < K; ++k) {
                P a = Arith<T>::val(row[tl + k * TS]);
                s0 += Arith<T>::negpart(a);
                s1 += Arith<T>::pospart(a);
            }
        }
    }
    for (int off = TS >> 1; off >= 1; off >>= 1) {
        s0 = s0 + __shfl_xor_sync(FULL, s0, off, TS);
        if (want1) s1 = s1 + __shfl_xor_sync(FULL, s1, off, TS);
    }
    v0 = s0;
    v1 = s1;
}

template <typename T, int R>
__device__ __forceinline__ void team_lrb(const T *row, int K, int TS, int tl, bool act, uint64_t (&mk)[4]) {
    uint64_t top[R];
#pragma unroll
    for (int r = 0; r < R; ++r) top[r] = ~0ull;
    if (act) {
        for (int k = 0; k < K; ++k) {
            const int pos = tl + k * TS;
            uint64_t t = ((uint64_t)Arith<T>::absbits(Arith<T>::val(row[pos])) << 32) | (uint32_t)pos;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (t < top[r]) { uint64_t x = top[r]; top[r] = t; t = x; }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        uint64_t m = top[0];
        for (int off = TS >> 1; off >= 1; off >>= 1) {
            uint64_t o = __shfl_xor_sync(FULL, (unsigned long long)m, off, TS);
            m = o < m ? o : m;
        }
        if (top[0] == m) {
#pragma unroll
            for (int q = 0; q + 1 < R; ++q) top[q] = top[q + 1];
            top[R - 1] = ~0ull;
        }
        mk[r] = m;
    }
}

// Load up to 16 values of a node row into registers (lane-per-path leaves).
template <typename T>
__device__ __forceinline__ void load16(const T *row, int nv, bool act, typename Arith<T>::P (&a)[16]) {
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = 0;
    if (!act) return;
    if (sizeof(T) == 4 && nv >= 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (4 * q < nv) {
                const float4 v = reinterpret_cast<const float4 *>(row)[q];
                a[4 * q] = v.x; a[4 * q + 1] = v.y; a[4 * q + 2] = v.z; a[4 * q + 3] = v.w;
            }
        }
    } else if (sizeof(T) == 1 && nv >= 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (4 * q < nv) {
                const uint32_t v = reinterpret_cast<const uint32_t *>(row)[q];
                a[4 * q] = (int)(int8_t)(v & 0xFF);
                a[4 * q + 1] = (int)(int8_t)((v >> 8) & 0xFF);
                a[4 * q + 2] = (int)(int8_t)((v >> 16) & 0xFF);
                a[4 * q + 3] = (int)(int8_t)(v >> 24);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (i < nv) a[i] = Arith<T>::val(row[i]);
    }
}

// Canonical pairwise tree sum of x[0..nv) in registers (nv <= 16, power of 2).
template <typename P>
__device__ __forceinline__ P reg_tree(P (&x)[16], int nv) {
#pragma unroll
    for (int h = 8; h >= 1; h >>= 1) {
        if (h < nv) {
#pragma unroll
            for (int i = 0; i < h; ++i) x[i] = x[i] + x[i + h];
        }
    }
    return x[0];
}

// ---------------------------------------------------------------------------
// Decode one frame: channel row -> payload bits, penalty, CRC flag, slot.
// Called by all W*32 threads of one frame group.
template <typename T, int W>
__device__ __forceinline__ void decode_frame(const CodeView &cv, uint8_t *S, uint8_t *Gs, const uint8_t *src,
                                             uint8_t *bits_row, float *pm_out, uint8_t *ok_out, int32_t *slot_out,
                                             int gidx, int gtid) {
    typedef typename Arith<T>::P PT;
    typedef typename Arith<T>::K KT;
    constexpr KT KINF = Arith<T>::KINF;
    constexpr int GT = W * 32;
    const Layout &lay = cv.lay;
    const int lane = gtid & 31;
    const int wig = gtid >> 5;
    const int n = cv.n, N = cv.N, L = cv.L;
    const int bwn = beta_words(n);

    T *chan = reinterpret_cast<T *>(S + lay.chan);
    KT *keys = reinterpret_cast<KT *>(S + lay.key);
    KT *survk = reinterpret_cast<KT *>(S + lay.surv);
    uint4 *cinfo = reinterpret_cast<uint4 *>(S + lay.cinfo);
    uint32_t *br = reinterpret_cast<uint32_t *>(S + lay.br);
    uint32_t *ubuf = reinterpret_cast<uint32_t *>(S + lay.ubuf);

    {
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
            const uint32_t opn = (o + 1 < cv.n_ops) ? __ldg(cv.ops + o + 1) : 0u;
            const uint32_t kind = op_kind(op);
            const int j = op_stage(op);
            const int dest = op_dest(op);
            const bool solo = op_solo(op);
            const bool runs = !solo || wig == 0;
            const int tid = solo ? lane : gtid;
            const int nthr = solo ? 32 : GT;
            uint8_t *idxc = S + lay.idx[cur];
            uint8_t *bidxc = S + lay.bidx[cur];

            if (kind == OP_F || kind == OP_G) {
                if (runs) {
                    // ---------------- F / G: stage j -> stage j-1 ----------------
                    const int jo = j - 1;
                    const int h = 1 << jo;
                    const T *inb = (j == n) ? chan : stage_ptr<T>(lay, S, Gs, j);
                    T *outb = stage_ptr<T>(lay, S, Gs, jo);
                    const bool isG = kind == OP_G;
                    const uint32_t *blb = reinterpret_cast<const uint32_t *>(S + lay.bl[jo]);
                    const int bwc = beta_words(jo);
                    if (sizeof(T) == 4 && h >= 4) {
                        const int lv = jo - 2;
                        const int total = La << lv;
                        for (int t = tid; t < total; t += nthr) {
                            const int p = t >> lv, v = t & ((1 << lv) - 1);
                            const float *in = reinterpret_cast<const float *>(inb) + (j == n ? 0 : ((int)idxc[p * 16 + j] << j));
                            const float4 a = reinterpret_cast<const float4 *>(in)[v];
                            const float4 b = reinterpret_cast<const float4 *>(in + h)[v];
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
                    } else if (sizeof(T) == 1 && h >= 16) {
                        const int lv = jo - 4;
                        const int total = La << lv;
                        for (int t = tid; t < total; t += nthr) {
                            const int p = t >> lv, v = t & ((1 << lv) - 1);
                            const int8_t *in = reinterpret_cast<const int8_t *>(inb) + (j == n ? 0 : ((int)idxc[p * 16 + j] << j));
                            const uint4 a = reinterpret_cast<const uint4 *>(in)[v];
                            const uint4 b = reinterpret_cast<const uint4 *>(in + h)[v];
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
                    } else if (sizeof(T) == 1 && h >= 4) {
                        const int lv = jo - 2;
                        const int total = La << lv;
                        for (int t = tid; t < total; t += nthr) {
                            const int p = t >> lv, v = t & ((1 << lv) - 1);
                            const int8_t *in = reinterpret_cast<const int8_t *>(inb) + (j == n ? 0 : ((int)idxc[p * 16 + j] << j));
                            const uint32_t a = reinterpret_cast<const uint32_t *>(in)[v];
                            const uint32_t b = reinterpret_cast<const uint32_t *>(in + h)[v];
                            uint32_t r;
                            if (isG) {
                                const int i = v << 2;
                                const uint32_t nb = blb[(int)bidxc[p * 16 + jo] * bwc + (i >> 5)] >> (i & 31);
                                r = g4(a, b, nb & 15u);
                            } else {
                                r = f4(a, b);
                            }
                            reinterpret_cast<uint32_t *>(reinterpret_cast<int8_t *>(outb) + (p << jo))[v] = r;
                        }
                    } else {
                        const int total = La << jo;
                        for (int t = tid; t < total; t += nthr) {
                            const int p = t >> jo, i = t & (h - 1);
                            const T *in = inb + (j == n ? 0 : ((int)idxc[p * 16 + j] << j));
                            T r;
                            if (isG) {
                                const uint32_t bb = (blb[(int)bidxc[p * 16 + jo] * bwc + (i >> 5)] >> (i & 31)) & 1u;
                                r = g_op(in[i], in[i + h], bb);
                            } else {
                                r = f_op(in[i], in[i + h]);
                            }
                            outb[(p << jo) + i] = r;
                        }
                    }
                    for (int t = tid; t < La; t += nthr) idxc[t * 16 + jo] = (uint8_t)t;
                }
            } else if (kind == OP_COMB) {
                if (runs) {
                    // ---------------- Combine: [beta_l ^ beta_r, beta_r] ----------------
                    const int jc = j - 1;
                    const int bwc = beta_words(jc);
                    const uint32_t *blb = reinterpret_cast<const uint32_t *>(S + lay.bl[jc]);
                    uint32_t *out = dest ? br : reinterpret_cast<uint32_t *>(S + lay.bl[j]);
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
            } else {
                // ---------------- leaves ----------------
                const int nv = 1 << j;
                T *stj = (j == n) ? chan : stage_ptr<T>(lay, S, Gs, j);
                PT *penc = reinterpret_cast<PT *>(S + lay.pen[cur]);
                uint32_t *bout = dest ? br : reinterpret_cast<uint32_t *>(S + lay.bl[j]);
                const int ostride = dest ? bwn : beta_words(j);
                const uint32_t wmask = nv >= 32 ? 0xffffffffu : ((1u << nv) - 1u);
                int C = 1;
                if (kind == OP_R1) C = nv == 1 ? 2 : 4;
                else if (kind == OP_REP) C = 2;
                else if (kind == OP_SPC) C = L == 2 ? 2 : 8;
                const int lc = C == 2 ? 1 : (C == 4 ? 2 : 3);
                const int nc = La * C;
                const int nxt = cur ^ 1;
                uint8_t *idxn = S + lay.idx[nxt];
                uint8_t *bidxn = S + lay.bidx[nxt];
                PT *penn = reinterpret_cast<PT *>(S + lay.pen[nxt]);

                if (nv <= 16) {
                    // ------- small leaf: warp 0, lane s = source path s -------
                    if (wig == 0) {
                        const int s = lane;
                        const bool act = s < La;
                        const T *row = stj + (j == n ? 0 : ((int)idxc[(act ? s : 0) * 16 + j] << j));
                        PT a[16];
                        load16<T>(row, nv, act, a);
                        const PT ps = act ? penc[s] : (PT)0;
                        if (kind == OP_R0) {
                            // Rate-0 (Sec. III-B): no fork, penalty += sum |min(a, 0)|, beta = 0.
                            PT x[16];
#pragma unroll
                            for (int i = 0; i < 16; ++i) x[i] = Arith<T>::negpart(a[i]);
                            const PT v0 = reg_tree(x, nv);
                            if (act) {
                                penc[s] = ps + v0;
                                bout[s * ostride] = 0u;
                                if (!dest) bidxc[s * 16 + j] = (uint8_t)s;
                            }
                        } else {
                            uint32_t hd = 0;
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (i < nv && a[i] < 0) hd |= 1u << i;
                            KT k[8];
#pragma unroll
                            for (int c = 0; c < 8; ++c) k[c] = KINF;
                            uint32_t mpos = 0, flag = 0;
                            if (kind == OP_REP) {
                                // Repetition (Sec. III-E): ML word listed first.
                                PT x0[16], x1[16];
#pragma unroll
                                for (int i = 0; i < 16; ++i) {
                                    x0[i] = Arith<T>::negpart(a[i]);
                                    x1[i] = Arith<T>::pospart(a[i]);
                                }
                                const PT p0 = reg_tree(x0, nv), p1 = reg_tree(x1, nv);
                                flag = (p0 <= p1) ? 0u : 1u;
                                k[0] = Arith<T>::mk(ps + (flag ? p1 : p0), s * 2 + 0);
                                k[1] = Arith<T>::mk(ps + (flag ? p0 : p1), s * 2 + 1);
                            } else {
                                // least reliable positions by (|a|, index): keys |a| << 4 | i
                                unsigned long long lk[4] = {~0ull, ~0ull, ~0ull, ~0ull};
#pragma unroll
                                for (int i = 0; i < 16; ++i) {
                                    if (i < nv) {
                                        unsigned long long v = ((unsigned long long)Arith<T>::absbits(a[i]) << 4) | (unsigned)i;
#pragma unroll
                                        for (int r = 0; r < 4; ++r) {
                                            if (v < lk[r]) { const unsigned long long t2 = lk[r]; lk[r] = v; v = t2; }
                                        }
                                    }
                                }
                                uint32_t b[4], m[4];
#pragma unroll
                                for (int r = 0; r < 4; ++r) {
                                    b[r] = (uint32_t)(lk[r] >> 4);
                                    m[r] = (uint32_t)(lk[r] & 15u);
                                }
                                mpos = m[0] | (m[1] << 4) | (m[2] << 8) | (m[3] << 12);
                                const PT a1 = Arith<T>::unabs(b[0]);
                                if (kind == OP_R1) {
                                    // Rate-1 (Sec. III-C): HD, HD^m1, HD^m2, HD^m1^m2.
                                    k[0] = Arith<T>::mk(ps, s * C + 0);
                                    k[1] = Arith<T>::mk(ps + a1, s * C + 1);
                                    if (C == 4) {
                                        const PT a2 = Arith<T>::unabs(b[1]);
                                        k[2] = Arith<T>::mk(ps + a2, s * C + 2);
                                        k[3] = Arith<T>::mk(ps + (a1 + a2), s * C + 3);
                                    }
                                } else {
                                    // SPC (Sec. III-D): ML = HD or HD^m1; ML ^ T, penalty from Eq. (9).
                                    flag = (__popc(hd) & 1u) ? 0u : 1u;   // q
                                    PT ar[4];
#pragma unroll
                                    for (int r = 0; r < 4; ++r) ar[r] = Arith<T>::unabs(b[r]);
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
                            // selection (Algorithm 1): keep the L smallest keys
                            const KT tau = (nc > L) ? warp_kth(k, C, L, lane) : KINF;
                            uint32_t sm = 0;
#pragma unroll
                            for (int r = 0; r < 8; ++r)
                                if (k[r] != KINF && k[r] <= tau) sm |= 1u << (Arith<T>::kidx(k[r]) & (uint32_t)(C - 1));
                            const int base = warp_excl_scan(__popc(sm), lane);
                            // commit: survivors of source s take slots in candidate order
#pragma unroll
                            for (int r = 0; r < 8; ++r) {
                                if (k[r] != KINF && k[r] <= tau) {
                                    const int c = (int)(Arith<T>::kidx(k[r]) & (uint32_t)(C - 1));
                                    const int t = base + __popc(sm & ((1u << c) - 1u));
                                    penn[t] = Arith<T>::kpen(k[r]);
                                    reinterpret_cast<uint4 *>(idxn)[t] = reinterpret_cast<const uint4 *>(idxc)[s];
                                    reinterpret_cast<uint4 *>(bidxn)[t] = reinterpret_cast<const uint4 *>(bidxc)[s];
                                    if (!dest) bidxn[t * 16 + j] = (uint8_t)t;
                                    uint32_t word;
                                    if (kind == OP_REP) {
                                        word = ((flag != 0u) != (c == 1)) ? wmask : 0u;
                                    } else {
                                        const uint32_t dm = (kind == OP_R1) ? (uint32_t)c : (spc_tmask(c) ^ (flag ? 0u : 1u));
                                        word = hd;
#pragma unroll
                                        for (int rr = 0; rr < 4; ++rr)
                                            if ((dm >> rr) & 1u) word ^= 1u << ((mpos >> (4 * rr)) & 15u);
                                    }
                                    bout[t * ostride] = word;
                                }
                            }
                        }
                    }
                } else {
                    // ------- large leaf: the group, a warp per source path -------
                    const int TS = 32;
                    const int K = nv >> 5;
                    const int rounds = (La + W - 1) / W;
                    for (int r = 0; r < rounds; ++r) {
                        const int s = r * W + wig;
                        const bool act = s < La;
                        T *row = stj + (j == n ? 0 : ((int)idxc[(act ? s : 0) * 16 + j] << j));
                        const PT ps = act ? penc[s] : (PT)0;
                        if (kind == OP_R0 || kind == OP_REP) {
                            PT v0, v1;
                            team_sums<T>(row, K, TS, lane, act, kind == OP_REP, v0, v1);
                            if (act && lane == 0) {
                                if (kind == OP_R0) {
                                    penc[s] = ps + v0;
                                } else {
                                    const bool one = !(v0 <= v1);
                                    keys[s * 2 + 0] = Arith<T>::mk(ps + (one ? v1 : v0), s * 2 + 0);
                                    keys[s * 2 + 1] = Arith<T>::mk(ps + (one ? v0 : v1), s * 2 + 1);
                                    cinfo[s] = make_uint4(0u, 0u, 0u, one ? 1u : 0u);
                                }
                            }
                        } else {
                            uint32_t hd = 0;
                            if (K == 1) hd = __ballot_sync(FULL, act && (Arith<T>::val(row[lane]) < 0));
                            uint64_t mk[4] = {~0ull, ~0ull, ~0ull, ~0ull};
                            if (kind == OP_R1) {
                                team_lrb<T, 2>(row, K, TS, lane, act, mk);
                                if (act && lane == 0) {
                                    const PT a1 = Arith<T>::unabs((uint32_t)(mk[0] >> 32));
                                    const PT a2 = Arith<T>::unabs((uint32_t)(mk[1] >> 32));
                                    keys[s * 4 + 0] = Arith<T>::mk(ps, s * 4 + 0);
                                    keys[s * 4 + 1] = Arith<T>::mk(ps + a1, s * 4 + 1);
                                    keys[s * 4 + 2] = Arith<T>::mk(ps + a2, s * 4 + 2);
                                    keys[s * 4 + 3] = Arith<T>::mk(ps + (a1 + a2), s * 4 + 3);
                                    cinfo[s] = make_uint4((uint32_t)mk[0] | ((uint32_t)mk[1] << 16), 0u, hd, 0u);
                                }
                            } else {
                                team_lrb<T, 4>(row, K, TS, lane, act, mk);
                                int cnt = 0;
                                if (act)
                                    for (int kk = 0; kk < K; ++kk) cnt += Arith<T>::val(row[lane + kk * TS]) < 0 ? 1 : 0;
                                for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(FULL, cnt, off);
                                if (act && lane == 0) {
                                    const uint32_t q = (cnt & 1) ? 0u : 1u;
                                    PT ar[4];
#pragma unroll
                                    for (int rr = 0; rr < 4; ++rr) ar[rr] = Arith<T>::unabs((uint32_t)(mk[rr] >> 32));
                                    for (int c = 0; c < C; ++c) {
                                        const uint32_t dm = spc_tmask(c) ^ (q ? 0u : 1u);
                                        PT inc = (PT)0;
                                        bool first = true;
#pragma unroll
                                        for (int rr = 0; rr < 4; ++rr)
                                            if ((dm >> rr) & 1u) { inc = first ? ar[rr] : inc + ar[rr]; first = false; }
                                        keys[s * C + c] = Arith<T>::mk(ps + inc, s * C + c);
                                    }
                                    cinfo[s] = make_uint4((uint32_t)mk[0] | ((uint32_t)mk[1] << 16),
                                                          (uint32_t)mk[2] | ((uint32_t)mk[3] << 16), hd, q);
                                }
                            }
                        }
                    }
                    if (kind == OP_R0) {
                        const int bw = beta_words(j);
                        for (int t = gtid; t < La * bw; t += GT) {
                            const int p = t / bw, w = t - p * bw;
                            bout[p * ostride + w] = 0u;
                        }
                        if (!dest)
                            for (int t = gtid; t < La; t += GT) bidxc[t * 16 + j] = (uint8_t)t;
                    } else {
                        gsync<W>(gidx);
                        // selection by warp 0 (Algorithm 1)
                        if (wig == 0) {
                            const int s = lane;
                            const bool act = s < La;
                            KT k[8];
#pragma unroll
                            for (int c = 0; c < 8; ++c) k[c] = (act && c < C) ? keys[s * C + c] : KINF;
                            if (C == 8) sort8(k);
                            const KT tau = (nc > L) ? warp_kth(k, C, L, lane) : KINF;
                            uint32_t sm = 0;
#pragma unroll
                            for (int r = 0; r < 8; ++r)
                                if (k[r] != KINF && k[r] <= tau) sm |= 1u << (Arith<T>::kidx(k[r]) & (uint32_t)(C - 1));
                            const int base = warp_excl_scan(__popc(sm), lane);
#pragma unroll
                            for (int r = 0; r < 8; ++r) {
                                if (k[r] != KINF && k[r] <= tau) {
                                    const int c = (int)(Arith<T>::kidx(k[r]) & (uint32_t)(C - 1));
                                    const int t = base + __popc(sm & ((1u << c) - 1u));
                                    survk[t] = k[r];
                                    penn[t] = Arith<T>::kpen(k[r]);
                                    reinterpret_cast<uint4 *>(idxn)[t] = reinterpret_cast<const uint4 *>(idxc)[s];
                                    reinterpret_cast<uint4 *>(bidxn)[t] = reinterpret_cast<const uint4 *>(bidxc)[s];
                                    if (!dest) bidxn[t * 16 + j] = (uint8_t)t;
                                }
                            }
                        }
                        gsync<W>(gidx);
                        const int nn = nc < L ? nc : L;
                        // candidate beta of every new slot (the group)
                        const int bw = beta_words(j);
                        if (kind == OP_REP) {
                            for (int t = gtid; t < nn * bw; t += GT) {
                                const int p = t / bw, w = t - p * bw;
                                const uint32_t ci = Arith<T>::kidx(survk[p]);
                                const int s = (int)(ci >> lc), c = (int)(ci & (uint32_t)(C - 1));
                                bout[p * ostride + w] = ((cinfo[s].w != 0u) != (c == 1)) ? wmask : 0u;
                            }
                        } else {
                            for (int q2 = wig; q2 < nn * bw; q2 += W) {
                                const int p = q2 / bw, w = q2 - p * bw;
                                const uint32_t ci = Arith<T>::kidx(survk[p]);
                                const int s = (int)(ci >> lc), c = (int)(ci & (uint32_t)(C - 1));
                                const T *row = stj + (j == n ? 0 : ((int)idxc[s * 16 + j] << j));
                                const uint32_t bal = __ballot_sync(FULL, Arith<T>::val(row[(w << 5) + lane]) < 0);
                                if (lane == 0) {
                                    const uint4 ci4 = cinfo[s];
                                    const uint32_t dm = (kind == OP_R1) ? (uint32_t)c : (spc_tmask(c) ^ (ci4.w ? 0u : 1u));
                                    const uint32_t m[4] = {ci4.x & 0xFFFFu, ci4.x >> 16, ci4.y & 0xFFFFu, ci4.y >> 16};
                                    uint32_t word = bal;
#pragma unroll
                                    for (int rr = 0; rr < 4; ++rr)
                                        if (((dm >> rr) & 1u) && (int)(m[rr] >> 5) == w) word ^= 1u << (m[rr] & 31u);
                                    bout[p * ostride + w] = word;
                                }
                            }
                        }
                    }
                }
                if (kind != OP_R0) {
                    La = nc < L ? nc : L;
                    cur = nxt;
                }
            }
            if (op_sync(op)) gsync<W>(gidx);
            else if (wig == 0) __syncwarp();
            op = opn;
        }
        gsync<W>(gidx);

        // ---------------- final pick (Sec. II-B) ----------------
        PT *penc = reinterpret_cast<PT *>(S + lay.pen[cur]);
        uint32_t *synb = reinterpret_cast<uint32_t *>(S + lay.cinfo);
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
                const unsigned long long o = __shfl_xor_sync(FULL, key, off);
                key = o < key ? o : key;
            }
            const int win = (int)(key & 0xFFu);
            const uint32_t okw = (uint32_t)(key >> 63) ^ 1u;
            // u = x G_N for the winner (natural-order butterflies)
            const uint32_t *xw = br + win * bwn;
            const int R = bwn > 32 ? bwn >> 5 : 1;
            uint32_t U[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int w = lane + 32 * r;
                U[r] = (r < R && w < bwn) ? xw[w] : 0u;
            }
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
}

// Plain form: one code, frames f = group, group + n_groups, ...
template <typename T, int W>
__global__ void __launch_bounds__(128) decode_kernel(const Params P) {
    constexpr int GT = W * 32;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int gidx = threadIdx.x / GT;
    const int gtid = threadIdx.x - gidx * GT;
    uint8_t *S = smem_raw + (size_t)gidx * P.cv.lay.bytes;
    const int ggid = blockIdx.x * P.groups_per_cta + gidx;
    const int ngroups = gridDim.x * P.groups_per_cta;
    uint8_t *Gs = P.scratch ? P.scratch + (size_t)ggid * P.cv.lay.gbytes : nullptr;
    const size_t nbytes = (size_t)P.cv.N * sizeof(T);
    for (uint32_t f = ggid; f < P.n_frames; f += ngroups) {
        decode_frame<T, W>(P.cv, S, Gs, reinterpret_cast<const uint8_t *>(P.llr) + (size_t)f * nbytes,
                           P.bits + (size_t)f * P.cv.kb, P.pm + f, P.ok ? P.ok + f : nullptr,
                           P.slot ? P.slot + f : nullptr, gidx, gtid);
    }
}

// Batched form: frames of several codes in one persistent launch. Groups take
// work items (ordered by decreasing cost) from a device counter; the code of
// an item is copied into the group's shared memory when it changes.
template <typename T, int W>
__global__ void __launch_bounds__(128) batch_kernel(const BatchParams B) {
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
    uint32_t loaded = 0xffffffffu;
    for (;;) {
        if (gtid == 0) *slot_word = atomicAdd(B.counter, 1u);
        gsync<W>(gidx);
        const uint32_t it = *slot_word;
        gsync<W>(gidx);
        if (it >= B.n_items) break;
        const BatchItem item = B.items[it];
        if (item.cls != loaded) {
            const uint32_t *srcw = reinterpret_cast<const uint32_t *>(B.classes + item.cls);
            uint32_t *dstw = reinterpret_cast<uint32_t *>(cvs);
            for (int t = gtid; t < (int)(sizeof(CodeView) / 4); t += GT) dstw[t] = srcw[t];
            loaded = item.cls;
            gsync<W>(gidx);
        }
        decode_frame<T, W>(*cvs, S, Gs, B.llr + item.llr_off, B.bits + item.bits_off, B.pm + item.frame,
                           B.ok ? B.ok + item.frame : nullptr, B.slot ? B.slot + item.frame : nullptr, gidx, gtid);
    }
}

template <typename T, int W>
cudaError_t launch_one(const LaunchShape &sh, const Params &p, int grid, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(decode_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sh.smem);
    if (e != cudaSuccess) return e;
    decode_kernel<T, W><<<grid, sh.threads, sh.smem, st>>>(p);
    return cudaGetLastError();
}

template <typename T, int W>
int occ_one(const LaunchShape &sh) {
    if (cudaFuncSetAttribute(decode_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem) !=
        cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, decode_kernel<T, W>, sh.threads, sh.smem) != cudaSuccess)
        return 0;
    return nb;
}

template <typename T, int W>
cudaError_t launch_batch_one(const BatchParams &b, int grid, uint32_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(batch_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    batch_kernel<T, W><<<grid, 128, smem, st>>>(b);
    return cudaGetLastError();
}

template <typename T, int W>
int occ_batch_one(uint32_t smem) {
    if (cudaFuncSetAttribute(batch_kernel<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel<T, W>, 128, smem) != cudaSuccess) return 0;
    return nb;
}

}  // namespace

cudaError_t launch_batch(int dtype, int warps, const BatchParams &b, int grid, uint32_t smem, cudaStream_t st) {
    if (dtype == 0) {
        if (warps == 1) return launch_batch_one<float, 1>(b, grid, smem, st);
        if (warps == 2) return launch_batch_one<float, 2>(b, grid, smem, st);
        if (warps == 4) return launch_batch_one<float, 4>(b, grid, smem, st);
    } else {
        if (warps == 1) return launch_batch_one<int8_t, 1>(b, grid, smem, st);
        if (warps == 2) return launch_batch_one<int8_t, 2>(b, grid, smem, st);
        if (warps == 4) return launch_batch_one<int8_t, 4>(b, grid, smem, st);
    }
    return cudaErrorInvalidValue;
}

int occupancy_batch(int dtype, int warps, uint32_t smem) {
    if (dtype == 0) {
        if (warps == 1) return occ_batch_one<float, 1>(smem);
        if (warps == 2) return occ_batch_one<float, 2>(smem);
        if (warps == 4) return occ_batch_one<float, 4>(smem);
    } else {
        if (warps == 1) return occ_batch_one<int8_t, 1>(smem);
        if (warps == 2) return occ_batch_one<int8_t, 2>(smem);
        if (warps == 4) return occ_batch_one<int8_t, 4>(smem);
    }
    return 0;
}

cudaError_t launch_decode(int dtype, const LaunchShape &sh, const Params &p, int grid, cudaStream_t st) {
    if (dtype == 0) {
        if (sh.warps == 1) return launch_one<float, 1>(sh, p, grid, st);
        if (sh.warps == 2) return launch_one<float, 2>(sh, p, grid, st);
        if (sh.warps == 4) return launch_one<float, 4>(sh, p, grid, st);
    } else {
        if (sh.warps == 1) return launch_one<int8_t, 1>(sh, p, grid, st);
        if (sh.warps == 2) return launch_one<int8_t, 2>(sh, p, grid, st);
        if (sh.warps == 4) return launch_one<int8_t, 4>(sh, p, grid, st);
    }
    return cudaErrorInvalidValue;
}

int occupancy(int dtype, const LaunchShape &sh) {
    if (dtype == 0) {
        if (sh.warps == 1) return occ_one<float, 1>(sh);
        if (sh.warps == 2) return occ_one<float, 2>(sh);
        if (sh.warps == 4) return occ_one<float, 4>(sh);
    } else {
        if (sh.warps == 1) return occ_one<int8_t, 1>(sh);
        if (sh.warps == 2) return occ_one<int8_t, 2>(sh);
        if (sh.warps == 4) return occ_one<int8_t, 4>(sh);
    }
    return 0;
}

}  // namespace polar
