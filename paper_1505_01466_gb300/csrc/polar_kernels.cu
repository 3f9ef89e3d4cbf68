// polar_kernels.cu -- list-CRC decoding of polar codes over the unrolled
// Fast-SSC tree, for GB300 (sm_103a).
//
// One frame is decoded by a group of W warps; a CTA holds 128 / (32 W)
// groups and every group loops over frames (persistent). All L paths of a
// frame advance through the same unrolled schedule in lockstep, so:
//
//  * alpha stage j holds one row of 2^j LLRs per physical slot. F and G
//    (Eq. (1), (2)) read stage j+1 through the path's index-table entry and
//    always write the path's own row of stage j: at that moment stage j is
//    dead for every path. A fork only copies the parent's index row -- the
//    lazy copy of Sec. IV-A -- never LLRs.
//  * beta is bit-packed. Left-child outputs (BL[j]) sit behind a second
//    index table (Sec. IV-B); the right-child / root output (BR) is consumed
//    by the Combine (Eq. (3)) that follows at once and needs none.
//  * a forking leaf (Sec. III-C..E) writes candidate keys
//    (penalty, source slot * C + candidate) to shared memory; when there are
//    more than L the group sorts them (bitonic) and the L smallest survive
//    (Algorithm 1). Survivors take slots in (source, candidate) order and
//    inherit their parent's index rows, penalty and candidate beta.
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

template <typename T> struct Arith;

template <> struct Arith<float> {
    typedef float P;
    static __device__ __forceinline__ uint32_t pkey(float p) { return __float_as_uint(p); }
    static __device__ __forceinline__ float punkey(uint32_t k) { return __uint_as_float(k); }
    static __device__ __forceinline__ float to_out(float p) { return p; }
    static __device__ __forceinline__ uint32_t absbits(float a) { return __float_as_uint(fabsf(a)); }
    static __device__ __forceinline__ float negpart(float a) { return a < 0.f ? -a : 0.f; }
    static __device__ __forceinline__ float pospart(float a) { return a > 0.f ? a : 0.f; }
    static __device__ __forceinline__ float val(float a) { return a; }
};

template <> struct Arith<int8_t> {
    typedef int P;
    static __device__ __forceinline__ uint32_t pkey(int p) { return (uint32_t)p; }
    static __device__ __forceinline__ int punkey(uint32_t k) { return (int)k; }
    static __device__ __forceinline__ float to_out(int p) { return (float)p; }
    static __device__ __forceinline__ uint32_t absbits(int a) { return (uint32_t)(a < 0 ? -a : a); }
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

__device__ __forceinline__ uint64_t mkkey(uint32_t pen_bits, uint32_t idx) {
    return ((uint64_t)pen_bits << 32) | idx;
}

__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int off, int width) {
    return __shfl_xor_sync(0xffffffffu, (unsigned long long)v, off, width);
}

// SPC candidate flips over the ranks of the four least reliable bits (bit r
// = rank r+1), in the candidate order {}, {1,2}, {1,3}, {1,4}, {2,3}, {2,4},
// {3,4}, {1,2,3,4}.
__device__ __forceinline__ uint32_t spc_tmask(int c) {
    return (0xFCA69530u >> (4 * c)) & 0xFu;
}

// Canonical sums of |min(a,0)| (v0) and |max(a,0)| (v1) over one node row
// held by a team of TS lanes (lane tl owns elements tl + TS*k). For float the
// in-lane levels run in place on the row (the leaf input is dead afterwards)
// and the cross-lane levels use an xor butterfly; int8 sums are exact.
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
        s0 = s0 + __shfl_xor_sync(0xffffffffu, s0, off, TS);
        if (want1) s1 = s1 + __shfl_xor_sync(0xffffffffu, s1, off, TS);
    }
    v0 = s0;
    v1 = s1;
}

// The R (<= 4) least reliable positions of a node row, ranked by
// (|a| ascending, index ascending): keys (|a| bits << 32 | position).
template <typename T, int R>
__device__ __forceinline__ void team_lrb(const T *row, int K, int TS, int tl, bool act,
                                         uint64_t (&mk)[4]) {
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
            uint64_t o = shfl_xor64(m, off, TS);
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

template <typename T, int W>
__global__ void __launch_bounds__(128) decode_kernel(const Params P) {
    typedef typename Arith<T>::P PT;
    constexpr int GT = W * 32;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const Layout &lay = P.lay;
    const int gidx = threadIdx.x / GT;
    const int gtid = threadIdx.x - gidx * GT;
    const int lane = threadIdx.x & 31;
    const int wig = gtid >> 5;
    uint8_t *S = smem_raw + (size_t)gidx * lay.bytes;
    const int ggid = blockIdx.x * P.groups_per_cta + gidx;
    const int ngroups = gridDim.x * P.groups_per_cta;
    uint8_t *Gs = P.scratch ? P.scratch + (size_t)ggid * lay.gbytes : nullptr;
    const int n = P.n, N = P.N, L = P.L, rowlen = n + 1;
    const int bwn = beta_words(n);

    T *chan = reinterpret_cast<T *>(S + lay.chan);
    uint64_t *keys = reinterpret_cast<uint64_t *>(S + lay.key);
    uint64_t *survk = reinterpret_cast<uint64_t *>(S + lay.surv);
    uint4 *cinfo = reinterpret_cast<uint4 *>(S + lay.cinfo);
    uint32_t *br = reinterpret_cast<uint32_t *>(S + lay.br);
    uint32_t *ubuf = reinterpret_cast<uint32_t *>(S + lay.ubuf);

    for (uint32_t f = ggid; f < P.n_frames; f += ngroups) {
        // ---------------- channel LLRs -> stage n ----------------
        {
            const size_t nbytes = (size_t)N * sizeof(T);
            const uint8_t *src = reinterpret_cast<const uint8_t *>(P.llr) + (size_t)f * nbytes;
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
        for (int t = gtid; t < L * rowlen; t += GT) {
            S[lay.idx[0] + t] = 0; S[lay.idx[1] + t] = 0;
            S[lay.bidx[0] + t] = 0; S[lay.bidx[1] + t] = 0;
        }
        int La = 1, cur = 0;
        if (gtid == 0) reinterpret_cast<PT *>(S + lay.pen[0])[0] = (PT)0;
        gsync<W>(gidx);

        for (int o = 0; o < P.n_ops; ++o) {
            const uint32_t op = __ldg(P.ops + o);
            const uint32_t kind = op_kind(op);
            const int j = op_stage(op);
            const int dest = op_dest(op);
            uint8_t *idxc = S + lay.idx[cur];
            uint8_t *bidxc = S + lay.bidx[cur];

            if (kind == OP_F || kind == OP_G) {
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
                    for (int t = gtid; t < total; t += GT) {
                        const int p = t >> lv, v = t & ((1 << lv) - 1);
                        const float *in = reinterpret_cast<const float *>(inb) + (j == n ? 0 : ((int)idxc[p * rowlen + j] << j));
                        const float4 a = reinterpret_cast<const float4 *>(in)[v];
                        const float4 b = reinterpret_cast<const float4 *>(in + h)[v];
                        float4 r;
                        if (isG) {
                            const int i = v << 2;
                            const uint32_t nb = blb[(int)bidxc[p * rowlen + jo] * bwc + (i >> 5)] >> (i & 31);
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
                    for (int t = gtid; t < total; t += GT) {
                        const int p = t >> lv, v = t & ((1 << lv) - 1);
                        const int8_t *in = reinterpret_cast<const int8_t *>(inb) + (j == n ? 0 : ((int)idxc[p * rowlen + j] << j));
                        const uint4 a = reinterpret_cast<const uint4 *>(in)[v];
                        const uint4 b = reinterpret_cast<const uint4 *>(in + h)[v];
                        uint4 r;
                        if (isG) {
                            const int i = v << 4;
                            const uint32_t nb = blb[(int)bidxc[p * rowlen + jo] * bwc + (i >> 5)] >> (i & 31);
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
                    for (int t = gtid; t < total; t += GT) {
                        const int p = t >> lv, v = t & ((1 << lv) - 1);
                        const int8_t *in = reinterpret_cast<const int8_t *>(inb) + (j == n ? 0 : ((int)idxc[p * rowlen + j] << j));
                        const uint32_t a = reinterpret_cast<const uint32_t *>(in)[v];
                        const uint32_t b = reinterpret_cast<const uint32_t *>(in + h)[v];
                        uint32_t r;
                        if (isG) {
                            const int i = v << 2;
                            const uint32_t nb = blb[(int)bidxc[p * rowlen + jo] * bwc + (i >> 5)] >> (i & 31);
                            r = g4(a, b, nb & 15u);
                        } else {
                            r = f4(a, b);
                        }
                        reinterpret_cast<uint32_t *>(reinterpret_cast<int8_t *>(outb) + (p << jo))[v] = r;
                    }
                } else {
                    const int total = La << jo;
                    for (int t = gtid; t < total; t += GT) {
                        const int p = t >> jo, i = t & (h - 1);
                        const T *in = inb + (j == n ? 0 : ((int)idxc[p * rowlen + j] << j));
                        T r;
                        if (isG) {
                            const uint32_t bb = (blb[(int)bidxc[p * rowlen + jo] * bwc + (i >> 5)] >> (i & 31)) & 1u;
                            r = g_op(in[i], in[i + h], bb);
                        } else {
                            r = f_op(in[i], in[i + h]);
                        }
                        outb[(p << jo) + i] = r;
                    }
                }
                for (int t = gtid; t < La; t += GT) idxc[t * rowlen + jo] = (uint8_t)t;
            } else if (kind == OP_COMB) {
                // ---------------- Combine: [beta_l ^ beta_r, beta_r] ----------------
                const int jc = j - 1;
                const int bwc = beta_words(jc);
                const uint32_t *blb = reinterpret_cast<const uint32_t *>(S + lay.bl[jc]);
                uint32_t *out = dest ? br : reinterpret_cast<uint32_t *>(S + lay.bl[j]);
                const int ostride = dest ? bwn : beta_words(j);
                if (jc >= 5) {
                    const int lw = jc - 5;
                    const int total = La << lw;
                    for (int t = gtid; t < total; t += GT) {
                        const int p = t >> lw, w = t & (bwc - 1);
                        const uint32_t l = blb[(int)bidxc[p * rowlen + jc] * bwc + w];
                        const uint32_t r = br[p * bwn + w];
                        uint32_t *o = out + p * ostride;
                        o[w] = l ^ r;
                        o[w + bwc] = r;
                    }
                } else {
                    const int h = 1 << jc;
                    const uint32_t m = (1u << h) - 1u;
                    for (int t = gtid; t < La; t += GT) {
                        const uint32_t l = blb[(int)bidxc[t * rowlen + jc]];
                        const uint32_t r = br[t * bwn];
                        out[t * ostride] = ((l ^ r) & m) | ((r & m) << h);
                    }
                }
                if (!dest)
                    for (int t = gtid; t < La; t += GT) bidxc[t * rowlen + j] = (uint8_t)t;
            } else {
                // ---------------- leaves ----------------
                const int nv = 1 << j;
                const int TS = nv < 32 ? nv : 32;
                const int tpw = 32 / TS;
                const int nteams = W * tpw;
                const int team = wig * tpw + lane / TS;
                const int tl = lane & (TS - 1);
                const int K = nv / TS;
                const int rounds = (La + nteams - 1) / nteams;
                T *stj = (j == n) ? chan : stage_ptr<T>(lay, S, Gs, j);
                PT *penc = reinterpret_cast<PT *>(S + lay.pen[cur]);
                uint32_t *bout = dest ? br : reinterpret_cast<uint32_t *>(S + lay.bl[j]);
                const int ostride = dest ? bwn : beta_words(j);
                const int bwj = beta_words(j);
                const uint32_t wmask = nv >= 32 ? 0xffffffffu : ((1u << nv) - 1u);

                if (kind == OP_R0) {
                    // Rate-0 (Sec. III-B): no fork, penalty += sum |min(a, 0)|, beta = 0.
                    for (int r = 0; r < rounds; ++r) {
                        const int s = r * nteams + team;
                        const bool act = s < La;
                        T *row = stj + (j == n ? 0 : ((int)idxc[(act ? s : 0) * rowlen + j] << j));
                        PT v0, v1;
                        team_sums<T>(row, K, TS, tl, act, false, v0, v1);
                        if (act && tl == 0) penc[s] = penc[s] + v0;
                    }
                    for (int t = gtid; t < La * bwj; t += GT) {
                        const int p = t / bwj, w = t - p * bwj;
                        bout[p * ostride + w] = 0u;
                    }
                    if (!dest)
                        for (int t = gtid; t < La; t += GT) bidxc[t * rowlen + j] = (uint8_t)t;
                    gsync<W>(gidx);
                    continue;
                }

                // ---- candidate generation (first pass of Algorithm 1) ----
                int C;
                if (kind == OP_R1) C = nv == 1 ? 2 : 4;
                else if (kind == OP_REP) C = 2;
                else C = L == 2 ? 2 : 8;
                const int lc = C == 2 ? 1 : (C == 4 ? 2 : 3);
                const int nc = La * C;
                int npad = 1;
                while (npad < nc) npad <<= 1;

                for (int r = 0; r < rounds; ++r) {
                    const int s = r * nteams + team;
                    const bool act = s < La;
                    T *row = stj + (j == n ? 0 : ((int)idxc[(act ? s : 0) * rowlen + j] << j));
                    const PT ps = act ? penc[s] : (PT)0;
                    if (kind == OP_REP) {
                        // Repetition (Sec. III-E): all-zero costs sum |min(a,0)|,
                        // all-one sum |max(a,0)|; the ML word is listed first.
                        PT v0, v1;
                        team_sums<T>(row, K, TS, tl, act, true, v0, v1);
                        if (act && tl == 0) {
                            const bool one = !(v0 <= v1);
                            keys[s * 2 + 0] = mkkey(Arith<T>::pkey(ps + (one ? v1 : v0)), s * 2 + 0);
                            keys[s * 2 + 1] = mkkey(Arith<T>::pkey(ps + (one ? v0 : v1)), s * 2 + 1);
                            cinfo[s] = make_uint4(0u, 0u, 0u, one ? 1u : 0u);
                        }
                    } else {
                        uint32_t hd = 0;
                        if (K == 1) {
                            const bool neg = act && (Arith<T>::val(row[tl]) < 0);
                            const uint32_t bal = __ballot_sync(0xffffffffu, neg);
                            hd = (bal >> (lane & ~(TS - 1))) & wmask;
                        }
                        uint64_t mk[4] = {~0ull, ~0ull, ~0ull, ~0ull};
                        if (kind == OP_R1) {
                            if (nv == 1) team_lrb<T, 1>(row, K, TS, tl, act, mk);
                            else team_lrb<T, 2>(row, K, TS, tl, act, mk);
                            if (act && tl == 0) {
                                // Rate-1 (Sec. III-C): HD, HD^m1, HD^m2, HD^m1^m2.
                                const PT a1 = Arith<T>::punkey((uint32_t)(mk[0] >> 32));
                                keys[s * C + 0] = mkkey(Arith<T>::pkey(ps), s * C + 0);
                                keys[s * C + 1] = mkkey(Arith<T>::pkey(ps + a1), s * C + 1);
                                if (C == 4) {
                                    const PT a2 = Arith<T>::punkey((uint32_t)(mk[1] >> 32));
                                    keys[s * C + 2] = mkkey(Arith<T>::pkey(ps + a2), s * C + 2);
                                    keys[s * C + 3] = mkkey(Arith<T>::pkey(ps + (a1 + a2)), s * C + 3);
                                }
                                cinfo[s] = make_uint4((uint32_t)mk[0] | ((uint32_t)(C == 4 ? (uint32_t)mk[1] : 0u) << 16), 0u, hd, 0u);
                            }
                        } else {
                            // SPC (Sec. III-D): ML = HD (even parity) or HD ^ m1;
                            // candidates ML ^ T, penalty = sum over bits differing from HD.
                            team_lrb<T, 4>(row, K, TS, tl, act, mk);
                            uint32_t par;
                            if (K == 1) {
                                par = __popc(hd) & 1u;
                            } else {
                                int cnt = 0;
                                if (act)
                                    for (int k = 0; k < K; ++k) cnt += Arith<T>::val(row[tl + k * TS]) < 0 ? 1 : 0;
                                for (int off = TS >> 1; off >= 1; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off, TS);
                                par = (uint32_t)cnt & 1u;
                            }
                            if (act && tl == 0) {
                                const uint32_t q = par == 0u ? 1u : 0u;
                                PT ar[4];
#pragma unroll
                                for (int rr = 0; rr < 4; ++rr) ar[rr] = Arith<T>::punkey((uint32_t)(mk[rr] >> 32));
                                for (int c = 0; c < C; ++c) {
                                    const uint32_t dm = spc_tmask(c) ^ (q ? 0u : 1u);
                                    PT inc = (PT)0;
                                    bool first = true;
#pragma unroll
                                    for (int rr = 0; rr < 4; ++rr) {
                                        if ((dm >> rr) & 1u) { inc = first ? ar[rr] : inc + ar[rr]; first = false; }
                                    }
                                    keys[s * C + c] = mkkey(Arith<T>::pkey(ps + inc), s * C + c);
                                }
                                cinfo[s] = make_uint4((uint32_t)mk[0] | ((uint32_t)mk[1] << 16),
                                                      (uint32_t)mk[2] | ((uint32_t)mk[3] << 16), hd, q);
                            }
                        }
                    }
                }
                for (int t = nc + gtid; t < npad; t += GT) keys[t] = ~0ull;
                gsync<W>(gidx);

                // ---- selection (second pass of Algorithm 1): keep the L smallest keys ----
                const uint64_t *src = keys;
                int nn = nc;
                if (nc > L) {
                    for (int kk = 2; kk <= npad; kk <<= 1) {
                        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                            for (int t = gtid; t < (npad >> 1); t += GT) {
                                const int i = ((t & ~(jj - 1)) << 1) | (t & (jj - 1));
                                const int l2 = i | jj;
                                const bool up = (i & kk) == 0;
                                const uint64_t x = keys[i], y = keys[l2];
                                if ((x > y) == up) { keys[i] = y; keys[l2] = x; }
                            }
                            gsync<W>(gidx);
                        }
                    }
                    // survivors, renumbered in (source, candidate) order
                    for (int t = gtid; t < L; t += GT) {
                        const uint64_t kt = keys[t];
                        const uint32_t ci = (uint32_t)kt;
                        int cnt = 0;
                        for (int u = 0; u < L; ++u) cnt += ((uint32_t)keys[u] < ci) ? 1 : 0;
                        survk[cnt] = kt;
                    }
                    gsync<W>(gidx);
                    src = survk;
                    nn = L;
                }

                // ---- commit: new slots inherit index rows, penalty and candidate beta ----
                const int nxt = cur ^ 1;
                uint8_t *idxn = S + lay.idx[nxt];
                uint8_t *bidxn = S + lay.bidx[nxt];
                PT *penn = reinterpret_cast<PT *>(S + lay.pen[nxt]);
                for (int t = gtid; t < nn; t += GT) {
                    const uint64_t kt = src[t];
                    const uint32_t ci = (uint32_t)kt;
                    const int s = (int)(ci >> lc), c = (int)(ci & (C - 1));
                    penn[t] = Arith<T>::punkey((uint32_t)(kt >> 32));
                    for (int e = 0; e < rowlen; ++e) {
                        idxn[t * rowlen + e] = idxc[s * rowlen + e];
                        bidxn[t * rowlen + e] = bidxc[s * rowlen + e];
                    }
                    if (!dest) bidxn[t * rowlen + j] = (uint8_t)t;
                    if (nv <= 32) {
                        const uint4 ci4 = cinfo[s];
                        uint32_t word;
                        if (kind == OP_REP) {
                            word = ((ci4.w != 0u) != (c == 1)) ? wmask : 0u;
                        } else if (kind == OP_R1) {
                            word = ci4.z;
                            if (c & 1) word ^= 1u << (ci4.x & 0xFFFFu);
                            if (c & 2) word ^= 1u << (ci4.x >> 16);
                        } else {
                            const uint32_t dm = spc_tmask(c) ^ (ci4.w ? 0u : 1u);
                            word = ci4.z;
                            if (dm & 1u) word ^= 1u << (ci4.x & 0xFFFFu);
                            if (dm & 2u) word ^= 1u << (ci4.x >> 16);
                            if (dm & 4u) word ^= 1u << (ci4.y & 0xFFFFu);
                            if (dm & 8u) word ^= 1u << (ci4.y >> 16);
                        }
                        bout[t * ostride] = word;
                    }
                }
                if (nv > 32) {
                    const int bw = nv >> 5;
                    if (kind == OP_REP) {
                        for (int t = gtid; t < nn * bw; t += GT) {
                            const int p = t / bw, w = t - p * bw;
                            const uint64_t kt = src[p];
                            const uint32_t ci = (uint32_t)kt;
                            const int s = (int)(ci >> lc), c = (int)(ci & (C - 1));
                            bout[p * ostride + w] = ((cinfo[s].w != 0u) != (c == 1)) ? 0xffffffffu : 0u;
                        }
                    } else {
                        for (int q2 = wig; q2 < nn * bw; q2 += W) {
                            const int p = q2 / bw, w = q2 - p * bw;
                            const uint64_t kt = src[p];
                            const uint32_t ci = (uint32_t)kt;
                            const int s = (int)(ci >> lc), c = (int)(ci & (C - 1));
                            const T *row = stj + (j == n ? 0 : ((int)idxc[s * rowlen + j] << j));
                            const uint32_t bal = __ballot_sync(0xffffffffu, Arith<T>::val(row[(w << 5) + lane]) < 0);
                            if (lane == 0) {
                                const uint4 ci4 = cinfo[s];
                                uint32_t dm;
                                if (kind == OP_R1) dm = (uint32_t)c;
                                else dm = spc_tmask(c) ^ (ci4.w ? 0u : 1u);
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
                cur = nxt;
                La = nn;
            }
            gsync<W>(gidx);
        }

        // ---------------- final pick (Sec. II-B) ----------------
        PT *penc = reinterpret_cast<PT *>(S + lay.pen[cur]);
        uint32_t *synb = reinterpret_cast<uint32_t *>(survk);
        if (P.crc_len > 0) {
            const int nbytes = N >> 3;
            for (int p = wig; p < La; p += W) {
                const uint8_t *xb = reinterpret_cast<const uint8_t *>(br + p * bwn);
                uint32_t acc = 0;
                for (int b = lane; b < nbytes; b += 32) acc ^= __ldg(P.syn + ((b << 8) | xb[b]));
                for (int off = 16; off >= 1; off >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, off);
                if (lane == 0) synb[p] = acc;
            }
        }
        gsync<W>(gidx);
        if (wig == 0) {
            uint64_t key = ~0ull;
            if (lane < La) {
                const bool okp = P.crc_len == 0 || synb[lane] == 0u;
                key = ((uint64_t)(okp ? 0u : 1u) << 63) | ((uint64_t)Arith<T>::pkey(penc[lane]) << 8) | (uint64_t)lane;
            }
            for (int off = 16; off >= 1; off >>= 1) {
                const uint64_t o = shfl_xor64(key, off, 32);
                key = o < key ? o : key;
            }
            const int win = (int)(key & 0xFFu);
            const uint32_t okw = (uint32_t)(key >> 63) ^ 1u;
            // u = x G_N for the winner (natural order butterflies)
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
                        const uint32_t v = __shfl_down_sync(0xffffffffu, U[r], d);
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
                P.pm[f] = Arith<T>::to_out(penc[win]);
                if (P.ok) P.ok[f] = (uint8_t)okw;
                if (P.slot) P.slot[f] = win;
            }
        }
        gsync<W>(gidx);
        for (int b = gtid; b < P.kb; b += GT) {
            uint32_t byte = 0;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int pos = 8 * b + t;
                if (pos < P.k) {
                    const uint32_t u = __ldg(P.info + pos);
                    byte |= ((ubuf[u >> 5] >> (u & 31u)) & 1u) << t;
                }
            }
            P.bits[(size_t)f * P.kb + b] = (uint8_t)byte;
        }
        gsync<W>(gidx);
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

}  // namespace

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
