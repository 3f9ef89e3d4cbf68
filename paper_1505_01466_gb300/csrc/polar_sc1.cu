// polar_sc1.cu -- list decoding with a list of one path, i.e. Fast-SSC
// decoding (Sec. II-D) of a polar-CRC code: the first stage of the adaptive
// decoder of Sec. V.
//
// With one path nothing forks and nothing is selected. Algorithm 1 with L = 1
// keeps the most likely candidate of every leaf: no other candidate has a
// smaller penalty, and a tie goes to candidate 0, which is that one. So
//  * Rate-0: beta = 0, penalty += sum |min(alpha, 0)|           (Eq. (10))
//  * Rate-1: beta = h(alpha), penalty unchanged                  (Sec. III-C)
//  * repetition: all zero iff P0 <= P1, penalty += that P        (Eq. (5))
//  * SPC: beta = h(alpha); when the parity fails, the least reliable bit
//    (smallest |alpha|, then lowest index) is flipped and penalty += its
//    |alpha|                                                    (Sec. III-D)
//
// One lane decodes one frame: a warp takes 32 frames and walks the unrolled
// schedule (Listing 2) once for all of them, every lane doing its own frame's
// work for each operation. There is no data-dependent control flow at L = 1,
// so the lanes never diverge, and the cost of interpreting an operation is
// shared by 32 frames. Storage is interleaved by lane:
//  * alpha stage j holds 2^j values per frame; value e of lane l sits in
//    32-bit word e * 32 + l of the stage (float32), or, for int8, four values
//    per word (value e in byte e & 3 of word (e >> 2) * 32 + l), so F and G
//    run four lanes of SIMD at a time. Every access of a warp touches 32
//    consecutive words: no bank conflicts in shared memory, one 128-byte line
//    in global memory.
//  * the stages go to the warp's shared memory up to a budget, the largest
//    ones to a per-warp region of global scratch (by default all of them:
//    the accesses are coalesced and the L1 cache keeps the hot low stages,
//    and without shared memory more warps fit per SM);
//  * beta is one bit-packed row of N bits per frame (word w of lane l at
//    w * 32 + l), in shared memory if the budget holds it: a leaf writes its bits at its position and
//    Combine (Eq. (3)) xors the right half into the left in place, so at the
//    end the row holds the codeword x;
//  * the channel row (stage n) is read from the caller's buffer;
//  * float codes with special nodes run the DROP instantiation: once the last
//    reader of a spilled stage (a G, or a leaf) is done, its lines are
//    discarded from L2, so that dead stages are not written back to DRAM
//    (the float kernel is bound by DRAM bandwidth). Plain SC decoding keeps
//    the other instantiation, which needs fewer registers.
//
// Float sums follow the pairwise tree s[i] = x[i] + x[i + n/2] (computed in
// the dead stage below the leaf); int8 LLRs use saturated G and exact
// integer penalties. These are the conventions of the list kernels, so the
// results equal theirs at L = 1.

#include <cstdint>
#include <type_traits>

#include "../../include/polar.h"
#include "polar_internal.h"

namespace polar {
namespace {

// Eq. (1), min-sum, and Eq. (2) on float32
__device__ __forceinline__ float f1(float a, float b) {
    const float m = fminf(fabsf(a), fabsf(b));
    return ((a < 0.f) != (b < 0.f)) ? -m : m;
}
__device__ __forceinline__ float g1(float a, float b, uint32_t beta) { return beta ? b - a : b + a; }

// Four int8 LLRs in one word: F = max(min(a, b), -max(a, b)); G with the four
// beta bits in nib (bit e -> byte e), saturated to [-127, 127].
__device__ __forceinline__ uint32_t f4(uint32_t a, uint32_t b) {
    return __vmaxs4(__vmins4(a, b), __vneg4(__vmaxs4(a, b)));
}
__device__ __forceinline__ uint32_t g4(uint32_t a, uint32_t b, uint32_t nib) {
    const uint32_t m = ((nib * 0x00204081u) & 0x01010101u) * 0xFFu;
    const uint32_t sa = (a & ~m) | (__vneg4(a) & m);
    return __vmaxs4(__vaddss4(b, sa), 0x81818181u);
}
__device__ __forceinline__ int byte_of(uint32_t w, int e) { return (int)(int8_t)((w >> (8 * (e & 3))) & 0xFFu); }

// Words of stages 0 .. j-1 a lane holds: stage j has 2^j values, one per
// word (float32) or four per word (int8, at least one word).
__host__ __device__ __forceinline__ int words_below(int j, int es) {
    if (es == 4) return (1 << j) - 1;
    return j <= 2 ? j : (1 << (j - 2)) + 1;
}

// Per-lane view of one warp's storage: stages below `split` in the warp's
// shared memory, the others in its global scratch, both interleaved by lane.
struct Lane {
    uint8_t *smem, *gmem;          // the warp's regions, offset to this lane (4 * lane)
    uint32_t *beta;                // beta row, offset to this lane (word w at beta[w * 32])
    int n, N, split, es;
    __device__ __forceinline__ uint8_t *stage(int j) const {
        return j < split ? smem + (size_t)words_below(j, es) * 128
                         : gmem + (size_t)(words_below(j, es) - words_below(split, es)) * 128;
    }
};

// The frame's channel row (stage n) and its alignment.
struct Chan {
    const uint8_t *row;
    bool vec;                      // 16-byte aligned rows: vector loads
};

// ---- float32 element access ----
__device__ __forceinline__ float ldf(const Lane &ln, const Chan &ch, int j, int e) {
    if (j == ln.n) return __ldg(reinterpret_cast<const float *>(ch.row) + e);
    return reinterpret_cast<const float *>(ln.stage(j))[e * 32];
}
__device__ __forceinline__ float4 ldf4(const Lane &ln, const Chan &ch, int j, int e) {   // values e .. e+3
    if (j == ln.n && ch.vec) return __ldg(reinterpret_cast<const float4 *>(ch.row + 4 * e));
    float4 r;
    r.x = ldf(ln, ch, j, e);
    r.y = ldf(ln, ch, j, e + 1);
    r.z = ldf(ln, ch, j, e + 2);
    r.w = ldf(ln, ch, j, e + 3);
    return r;
}

// ---- int8 word access: word w = values 4w .. 4w+3 (a stage of fewer than
// four values uses the low bytes of word 0); the channel reads -128 as -127 ----
__device__ __forceinline__ uint32_t ldw(const Lane &ln, const Chan &ch, int j, int w) {
    if (j == ln.n) {
        uint32_t v;
        if (ch.vec) {
            v = __ldg(reinterpret_cast<const uint32_t *>(ch.row) + w);
        } else {
            const uint8_t *p = ch.row + 4 * w;
            v = (uint32_t)__ldg(p) | ((uint32_t)__ldg(p + 1) << 8) | ((uint32_t)__ldg(p + 2) << 16) |
                ((uint32_t)__ldg(p + 3) << 24);
        }
        return __vmaxs4(v, 0x81818181u);
    }
    return reinterpret_cast<const uint32_t *>(ln.stage(j))[w * 32];
}

__device__ __forceinline__ uint32_t beta_bits(const Lane &ln, int pos) {   // bits pos .. pos+31 (pos % 32 + span <= 32)
    return ln.beta[(pos >> 5) * 32] >> (pos & 31);
}
// Write nb (< 32) bits at position s (within one word) or whole words.
__device__ __forceinline__ void put_bits(const Lane &ln, int s, int nb, uint32_t bits) {
    if (nb >= 32) {
        ln.beta[(s >> 5) * 32] = bits;
    } else {
        const uint32_t m = ((1u << nb) - 1u) << (s & 31);
        uint32_t &w = ln.beta[(s >> 5) * 32];
        w = (w & ~m) | ((bits << (s & 31)) & m);
    }
}

// ---- F / G (Eq. (1), (2)) of a node of stage j starting at bit s ----------
template <bool IS_G>
__device__ __forceinline__ void fg_f32(const Lane &ln, const Chan &ch, int j, int s) {
    const int h = 1 << (j - 1);
    float *out = reinterpret_cast<float *>(ln.stage(j - 1));
    if (h >= 4) {
#pragma unroll 2
        for (int e = 0; e < h; e += 4) {
            const float4 a = ldf4(ln, ch, j, e), b = ldf4(ln, ch, j, e + h);
            if (IS_G) {
                const uint32_t nib = beta_bits(ln, s + e);
                out[e * 32] = g1(a.x, b.x, nib & 1u);
                out[(e + 1) * 32] = g1(a.y, b.y, (nib >> 1) & 1u);
                out[(e + 2) * 32] = g1(a.z, b.z, (nib >> 2) & 1u);
                out[(e + 3) * 32] = g1(a.w, b.w, (nib >> 3) & 1u);
            } else {
                out[e * 32] = f1(a.x, b.x);
                out[(e + 1) * 32] = f1(a.y, b.y);
                out[(e + 2) * 32] = f1(a.z, b.z);
                out[(e + 3) * 32] = f1(a.w, b.w);
            }
        }
    } else {
        const uint32_t nib = IS_G ? beta_bits(ln, s) : 0u;
        for (int e = 0; e < h; ++e) {
            const float a = ldf(ln, ch, j, e), b = ldf(ln, ch, j, e + h);
            out[e * 32] = IS_G ? g1(a, b, (nib >> e) & 1u) : f1(a, b);
        }
    }
}

template <bool IS_G>
__device__ __forceinline__ void fg_i8(const Lane &ln, const Chan &ch, int j, int s) {
    const int h = 1 << (j - 1);
    uint32_t *out = reinterpret_cast<uint32_t *>(ln.stage(j - 1));
    if (h >= 4) {
        const int hw = h >> 2;
#pragma unroll 4
        for (int w = 0; w < hw; ++w) {
            const uint32_t a = ldw(ln, ch, j, w), b = ldw(ln, ch, j, w + hw);
            out[w * 32] = IS_G ? g4(a, b, beta_bits(ln, s + 4 * w) & 15u) : f4(a, b);
        }
    } else {
        // two values (j = 2) or one (j = 1) in the low bytes of one word
        const uint32_t x = ldw(ln, ch, j, 0);
        const uint32_t b = x >> (8 * h);
        const uint32_t keep = h == 2 ? 0xFFFFu : 0xFFu;
        out[0] = (IS_G ? g4(x, b, beta_bits(ln, s) & ((1u << h) - 1u)) : f4(x, b)) & keep;
    }
}

// ---- Combine (Eq. (3)) in place on the beta row ----
__device__ __forceinline__ void comb(const Lane &ln, int j, int s) {
    const int h = 1 << (j - 1);
    if (h >= 32) {
        for (int w = 0; w < (h >> 5); ++w) ln.beta[((s >> 5) + w) * 32] ^= ln.beta[(((s + h) >> 5) + w) * 32];
    } else {
        uint32_t &W = ln.beta[(s >> 5) * 32];
        W ^= (W >> h) & (((1u << h) - 1u) << (s & 31));
    }
}

// ---- leaves ----------------------------------------------------------------
// Pairwise tree sum of |min(a, 0)| (neg) or max(a, 0) (!neg) over the nv =
// 2^j values of stage j, in the dead stage j - 1 (float32).
__device__ float tsum_f32(const Lane &ln, const Chan &ch, int j, bool neg) {
    auto t = [neg](float x) { return neg ? (x < 0.f ? -x : 0.f) : (x > 0.f ? x : 0.f); };
    if (j == 0) return t(ldf(ln, ch, 0, 0));
    const int h = 1 << (j - 1);
    float *scr = reinterpret_cast<float *>(ln.stage(j - 1));
    for (int i = 0; i < h; ++i) scr[i * 32] = t(ldf(ln, ch, j, i)) + t(ldf(ln, ch, j, i + h));
    for (int m = h; m > 1; m >>= 1) {
        const int hh = m >> 1;
        for (int i = 0; i < hh; ++i) scr[i * 32] = scr[i * 32] + scr[(i + hh) * 32];
    }
    return scr[0];
}

// Integer sums are exact in any order (int8): sums of |min(a,0)| and max(a,0).
__device__ void isums(const Lane &ln, const Chan &ch, int j, int &s0, int &s1) {
    const int nv = 1 << j;
    int a0 = 0, a1 = 0;
    for (int w = 0; w < (nv + 3) / 4; ++w) {
        const uint32_t x = ldw(ln, ch, j, w);
        const int cnt = nv < 4 ? nv : 4;
        for (int b = 0; b < cnt; ++b) {
            const int v = byte_of(x, b);
            a0 += v < 0 ? -v : 0;
            a1 += v > 0 ? v : 0;
        }
    }
    s0 = a0;
    s1 = a1;
}

// Hard decisions of values c*32 .. c*32 + cnt - 1 of stage j as one word.
template <typename T>
__device__ __forceinline__ uint32_t hd_chunk(const Lane &ln, const Chan &ch, int j, int c, int cnt) {
    uint32_t bits = 0;
    if (sizeof(T) == 4) {
        if (cnt >= 4) {
            for (int e = 0; e < cnt; e += 4) {
                const float4 v = ldf4(ln, ch, j, 32 * c + e);
                bits |= ((uint32_t)(v.x < 0.f) | ((uint32_t)(v.y < 0.f) << 1) | ((uint32_t)(v.z < 0.f) << 2) |
                         ((uint32_t)(v.w < 0.f) << 3)) << e;
            }
        } else {
            for (int e = 0; e < cnt; ++e) bits |= (uint32_t)(ldf(ln, ch, j, 32 * c + e) < 0.f) << e;
        }
    } else {
        for (int w = 0; w < (cnt + 3) / 4; ++w) {
            const uint32_t t = (ldw(ln, ch, j, 8 * c + w) >> 7) & 0x01010101u;     // sign bit of each byte
            bits |= (((t * 0x01020408u) >> 24) & 0xFu) << (4 * w);
        }
        if (cnt < 32) bits &= (1u << cnt) - 1u;
    }
    return bits;
}

// |value| and position of the least reliable value (smallest |a|, lowest index).
template <typename T>
__device__ __forceinline__ void lrb1(const Lane &ln, const Chan &ch, int j, uint32_t &best_abs, int &best_e) {
    const int nv = 1 << j;
    uint32_t ba = 0xffffffffu;
    int be = 0;
    if (sizeof(T) == 4) {
        for (int e = 0; e < nv; e += 4) {
            const float4 v = ldf4(ln, ch, j, e);
            const uint32_t x0 = __float_as_uint(fabsf(v.x)), x1 = __float_as_uint(fabsf(v.y));
            const uint32_t x2 = __float_as_uint(fabsf(v.z)), x3 = __float_as_uint(fabsf(v.w));
            if (x0 < ba) { ba = x0; be = e; }
            if (x1 < ba) { ba = x1; be = e + 1; }
            if (x2 < ba) { ba = x2; be = e + 2; }
            if (x3 < ba) { ba = x3; be = e + 3; }
        }
    } else {
        for (int w = 0; w < nv / 4; ++w) {
            const uint32_t x = ldw(ln, ch, j, w);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int v = byte_of(x, b);
                const uint32_t a = (uint32_t)(v < 0 ? -v : v);
                if (a < ba) { ba = a; be = 4 * w + b; }
            }
        }
    }
    best_abs = ba;
    best_e = be;
}

template <typename T, typename PT>
__device__ __forceinline__ void leaf(const Lane &ln, const Chan &ch, int kind, int j, int s, PT &pen) {
    const int nv = 1 << j;
    const int nch = nv >= 32 ? nv >> 5 : 1;
    const int cnt = nv >= 32 ? 32 : nv;
    if (kind == OP_R0) {                                               // Eq. (10)
        if (sizeof(T) == 4) {
            pen = pen + (PT)tsum_f32(ln, ch, j, true);
        } else {
            int s0, s1;
            isums(ln, ch, j, s0, s1);
            pen = pen + (PT)s0;
        }
        for (int c = 0; c < nch; ++c) put_bits(ln, s + 32 * c, cnt, 0u);
    } else if (kind == OP_R1) {                                        // Sec. III-C
        for (int c = 0; c < nch; ++c) put_bits(ln, s + 32 * c, cnt, hd_chunk<T>(ln, ch, j, c, cnt));
    } else if (kind == OP_REP) {                                       // Eq. (5), ties to all zero
        bool one;
        if (sizeof(T) == 4) {
            const float p0 = tsum_f32(ln, ch, j, true);
            const float p1 = tsum_f32(ln, ch, j, false);
            one = !(p0 <= p1);
            pen = pen + (PT)(one ? p1 : p0);
        } else {
            int s0, s1;
            isums(ln, ch, j, s0, s1);
            one = !(s0 <= s1);
            pen = pen + (PT)(one ? s1 : s0);
        }
        for (int c = 0; c < nch; ++c) put_bits(ln, s + 32 * c, cnt, one ? 0xffffffffu : 0u);
    } else {                                                           // SPC, Sec. III-D
        uint32_t par = 0;
        for (int c = 0; c < nch; ++c) {
            const uint32_t b = hd_chunk<T>(ln, ch, j, c, cnt);
            par ^= (uint32_t)__popc(b);
            put_bits(ln, s + 32 * c, cnt, b);
        }
        if (par & 1u) {
            uint32_t ba;
            int be;
            lrb1<T>(ln, ch, j, ba, be);
            ln.beta[((s + be) >> 5) * 32] ^= 1u << ((s + be) & 31);
            if (sizeof(T) == 4) pen = pen + (PT)__uint_as_float(ba);
            else pen = pen + (PT)ba;
        }
    }
}

template <typename T, bool DROP>
__global__ void __launch_bounds__(kSc1Threads) sc1_kernel(const Sc1Params p) {
    static_assert(!DROP || sizeof(T) == 4, "stages are dropped for float only");
    typedef typename std::conditional<sizeof(T) == 4, float, int>::type PT;   // penalty: exact int for int8
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t wpc = blockDim.x >> 5;
    const int es = sizeof(T);
    Lane ln;
    ln.n = p.n;
    ln.N = 1 << p.n;
    ln.es = es;
    ln.split = p.split;
    ln.smem = smem_raw + (size_t)warp * p.warp_bytes + 4 * lane;
    uint8_t *gwarp = p.scratch ? p.scratch + (size_t)(blockIdx.x * wpc + warp) * p.warp_gbytes : nullptr;
    ln.gmem = gwarp ? gwarp + 4 * lane : nullptr;
    ln.beta = reinterpret_cast<uint32_t *>((p.beta_smem ? smem_raw + (size_t)warp * p.warp_bytes : gwarp) +
                                           p.beta_off) + lane;
    const int N = ln.N;
    const int bwn = N >= 32 ? N >> 5 : 1;
    const uint32_t count = p.frame_idx ? *p.frame_cnt : p.n_frames;
    const bool vec = (reinterpret_cast<uintptr_t>(p.llr) & (es == 4 ? 15u : 3u)) == 0;
    for (uint32_t base = (blockIdx.x * wpc + warp) * 32u; base < count; base += gridDim.x * wpc * 32u) {
        const uint32_t i = base + (uint32_t)lane;
        const bool valid = i < count;
        const uint32_t ic = valid ? i : count - 1u;                  // idle lanes redo the last frame, unwritten
        const uint32_t f = p.frame_idx ? p.frame_idx[ic] : ic;
        Chan ch;
        ch.row = reinterpret_cast<const uint8_t *>(p.llr) + (size_t)f * N * es;
        ch.vec = vec;
        PT pen = 0;
        for (int w = 0; w < bwn; ++w) ln.beta[w * 32] = 0u;
        for (int o = 0; o < p.n_ops; ++o) {
            const uint32_t op = __ldg(p.ops + o);                     // the same for every lane
            const int kind = (int)(op & 15u), j = (int)((op >> 4) & 15u), s = (int)(op >> 8);
            if (kind == OP_F) {
                if (es == 4) fg_f32<false>(ln, ch, j, s); else fg_i8<false>(ln, ch, j, s);
            } else if (kind == OP_G) {
                if (es == 4) fg_f32<true>(ln, ch, j, s); else fg_i8<true>(ln, ch, j, s);
            } else if (kind == OP_COMB) {
                comb(ln, j, s);
            } else {
                leaf<T, PT>(ln, ch, kind, j, s, pen);
            }
            // DROP (float, node sets with special nodes): after the last reader
            // of stage j (G, or a leaf) its lines are dead until an F or G
            // rewrites them; drop them from L2 so that they are never written
            // back (this kernel is bound by DRAM bandwidth, much of it the
            // write-back of spilled stages)
            if (DROP && gwarp && j < p.n && j >= p.split && kind != OP_F && kind != OP_COMB) {
                uint8_t *dead = gwarp + (size_t)(words_below(j, es) - words_below(p.split, es)) * 128;
                if ((reinterpret_cast<uintptr_t>(dead) & 127u) == 0) {
                    __syncwarp();
                    for (int q = lane; q < (1 << j); q += 32)
                        asm volatile("discard.global.L2 [%0], 128;" ::"l"(dead + (size_t)q * 128) : "memory");
                    __syncwarp();
                }
            }
        }

        // ---------------- final pick (Sec. II-B) ----------------
        // CRC: the syndrome of the codeword x (the beta row), byte by byte
        uint32_t acc = 0;
        if (p.crc_len > 0) {
            for (int w = 0; w < (N >> 5 ? N >> 5 : 1); ++w) {
                const uint32_t x = ln.beta[w * 32];
                const int nb = N >= 32 ? 4 : N / 8;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (b < nb) acc ^= __ldg(p.syn + (((4 * w + b) << 8) | ((x >> (8 * b)) & 0xFFu)));
            }
        }
        // u = x G_N (natural-order butterflies) unless the code is systematic
        if (!p.systematic) {
            const uint32_t M[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
            for (int w = 0; w < bwn; ++w) {
                uint32_t u = ln.beta[w * 32];
#pragma unroll
                for (int e = 0; e < 5; ++e)
                    if ((1 << e) < N) u ^= (u >> (1 << e)) & M[e];
                ln.beta[w * 32] = u;
            }
            for (int d = 1; d < bwn; d <<= 1)
                for (int w = 0; w < bwn; ++w)
                    if (!(w & d)) ln.beta[w * 32] ^= ln.beta[(w + d) * 32];
        }
        if (valid) {
            uint8_t *row = p.bits + (size_t)f * p.kb;
            for (int b = 0; b < p.kb; ++b) {
                uint32_t byte = 0;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int pos = 8 * b + t;
                    if (pos < p.k) {
                        const uint32_t u = __ldg(p.info + pos);
                        byte |= ((ln.beta[(u >> 5) * 32] >> (u & 31u)) & 1u) << t;
                    }
                }
                row[b] = (uint8_t)byte;
            }
            p.pm[f] = (float)pen;
            if (p.ok) p.ok[f] = (uint8_t)(p.crc_len == 0 || acc == 0u);
            if (p.slot) p.slot[f] = 0;
        }
    }
}

}  // namespace

// Layout of one warp (32 frames) for a shared-memory budget: the beta rows
// go to shared memory if they fit, then alpha stages 0 .. split-1 while the
// total fits; everything else (higher stages, and the beta rows if they did
// not fit) to the warp's global scratch, stages first.
void sc1_layout(int n, int es, uint32_t budget, Sc1Layout *lay) {
    const int N = 1 << n;
    const uint32_t beta_bytes = (uint32_t)(N >= 32 ? N / 32 : 1) * 128u;
    lay->beta_smem = beta_bytes <= budget ? 1 : 0;
    int split = 0;
    if (lay->beta_smem)
        while (split < n && (uint32_t)words_below(split + 1, es) * 128u + beta_bytes <= budget) ++split;
    lay->split = split;
    const uint32_t sb = (uint32_t)words_below(split, es) * 128u;
    const uint64_t gb = (uint64_t)(words_below(n, es) - words_below(split, es)) * 128u;
    lay->warp_bytes = sb + (lay->beta_smem ? beta_bytes : 0u);
    lay->beta_off = lay->beta_smem ? sb : (uint32_t)gb;     // in shared memory, or in scratch after the stages
    lay->warp_gbytes = gb + (lay->beta_smem ? 0u : beta_bytes);
}

int occupancy_sc1(int dtype, uint32_t warp_bytes, int warps, bool drop) {
    const int smem = warps * (int)warp_bytes;
    const void *fn = dtype == POLAR_LLR_I8 ? (const void *)sc1_kernel<int8_t, false>
                                           : (drop ? (const void *)sc1_kernel<float, true> : (const void *)sc1_kernel<float, false>);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, 32 * warps, smem) != cudaSuccess) return 0;
    return blocks;
}

cudaError_t launch_sc1(int dtype, const Sc1Params &p, int grid, int warps, cudaStream_t st) {
    const int smem = warps * (int)p.warp_bytes;
    if (dtype == POLAR_LLR_I8) {
        cudaFuncSetAttribute(sc1_kernel<int8_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        sc1_kernel<int8_t, false><<<grid, 32 * warps, smem, st>>>(p);
    } else if (p.drop) {
        cudaFuncSetAttribute(sc1_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        sc1_kernel<float, true><<<grid, 32 * warps, smem, st>>>(p);
    } else {
        cudaFuncSetAttribute(sc1_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        sc1_kernel<float, false><<<grid, 32 * warps, smem, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace polar
