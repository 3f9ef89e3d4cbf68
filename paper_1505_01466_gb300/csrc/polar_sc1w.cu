// polar_sc1w.cu -- list decoding with a list of one path (Fast-SSC decoding,
// Sec. II-D, of a polar-CRC code: the first stage of the adaptive decoder of
// Sec. V) for small batches: one warp per frame, the lanes over the elements
// of a node. polar_sc1.cu gives each frame one lane, which is the faster way
// to decode many frames; a frame alone there walks the whole schedule on one
// lane, and here on 32.
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
// One warp decodes one frame, and the warps of the grid take frames in turn.
//  * Alpha stages 6..n-1 sit in the warp's shared memory (stage j at element
//    offset 2^j); the channel row is read from global memory by the two
//    operations at the root (a code whose root is itself a leaf copies it to
//    shared memory first).
//  * Every node of at most 32 bits runs in registers: stage 5 in one register
//    (element e in lane e), stages 0..4 together in another (stage j in lanes
//    2^j .. 2^(j+1)-1), F and G by two warp shuffles each, and the node's 32
//    beta bits in one word.
//  * Beta is one bit-packed row of N bits in shared memory: a leaf writes its
//    bits at its own position and Combine (Eq. (3)) xors the right half into
//    the left in place, so at the end the row holds the codeword x.
//
// Float sums follow the pairwise tree s[i] = x[i] + x[i + n/2]; int8 LLRs use
// saturated G and exact integer penalties. These are the conventions of the
// list kernels, so the results equal theirs at L = 1.

#include <cstdint>

#include "../../include/polar.h"
#include "polar_internal.h"

namespace polar {
namespace {

constexpr uint32_t FULL = 0xffffffffu;

template <typename T> struct A1;

template <> struct A1<float> {
    typedef float V;
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ float ldch(const float *p) { return __ldg(p); }
    // Eq. (1), min-sum, sign by comparison
    static __device__ __forceinline__ float f(float a, float b) {
        const float m = fminf(fabsf(a), fabsf(b));
        return ((a < 0.f) != (b < 0.f)) ? -m : m;
    }
    // Eq. (2)
    static __device__ __forceinline__ float g(float a, float b, uint32_t beta) { return beta ? b - a : b + a; }
    static __device__ __forceinline__ float st(float v) { return v; }
    static __device__ __forceinline__ uint32_t absbits(float a) { return __float_as_uint(fabsf(a)); }
    static __device__ __forceinline__ float absv(float a) { return fabsf(a); }
    static __device__ __forceinline__ float unabs(uint32_t b) { return __uint_as_float(b); }
    static __device__ __forceinline__ float negpart(float a) { return a < 0.f ? -a : 0.f; }
    static __device__ __forceinline__ float pospart(float a) { return a > 0.f ? a : 0.f; }
};

template <> struct A1<int8_t> {
    typedef int V;
    static __device__ __forceinline__ int ld(const int8_t *p) { return *p; }
    // -128 is read as -127
    static __device__ __forceinline__ int ldch(const int8_t *p) {
        const int v = __ldg(reinterpret_cast<const signed char *>(p));
        return v < -127 ? -127 : v;
    }
    static __device__ __forceinline__ int f(int a, int b) {
        const int m = min(abs(a), abs(b));
        return ((a < 0) != (b < 0)) ? -m : m;
    }
    static __device__ __forceinline__ int g(int a, int b, uint32_t beta) {
        const int r = beta ? b - a : b + a;
        return max(-127, min(127, r));
    }
    static __device__ __forceinline__ int8_t st(int v) { return (int8_t)v; }
    static __device__ __forceinline__ uint32_t absbits(int a) { return (uint32_t)abs(a); }
    static __device__ __forceinline__ int absv(int a) { return abs(a); }
    static __device__ __forceinline__ int unabs(uint32_t b) { return (int)b; }
    static __device__ __forceinline__ int negpart(int a) { return a < 0 ? -a : 0; }
    static __device__ __forceinline__ int pospart(int a) { return a > 0 ? a : 0; }
};

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

__device__ __forceinline__ uint32_t beta_bit(const uint32_t *bw, int pos) {
    return (bw[pos >> 5] >> (pos & 31)) & 1u;
}

// Write the bits of a node of nv bits at position s; lane l holds element
// l + 32 c of chunk c in its predicate.
__device__ __forceinline__ void put_chunk(uint32_t *bw, int s, int nv, int c, bool bit, int lane) {
    const uint32_t b = __ballot_sync(FULL, bit);
    if (lane == 0) {
        if (nv >= 32) {
            bw[(s >> 5) + c] = b;
        } else {
            const uint32_t m = ((1u << nv) - 1u) << (s & 31);
            uint32_t &w = bw[s >> 5];
            w = (w & ~m) | ((b << (s & 31)) & m);
        }
    }
}

// Pairwise tree sum of |min(a,0)| (neg) or max(a,0) (!neg) over a[0..nv),
// returned to every lane. Sums of more than 32 terms use scr (nv/2 floats).
__device__ float tree_sum(const float *a, int nv, bool neg, float *scr, int lane) {
    auto t = [neg](float x) { return neg ? (x < 0.f ? -x : 0.f) : (x > 0.f ? x : 0.f); };
    float v;
    if (nv > 32) {
        const int h = nv >> 1;
        for (int i = lane; i < h; i += 32) scr[i] = t(a[i]) + t(a[i + h]);
        __syncwarp();
        for (int m = h; m > 32; m >>= 1) {
            const int hh = m >> 1;
            for (int i = lane; i < hh; i += 32) scr[i] = scr[i] + scr[i + hh];
            __syncwarp();
        }
        v = scr[lane];
        __syncwarp();
        nv = 32;
    } else {
        v = lane < nv ? t(a[lane]) : 0.f;
    }
    for (int h = nv >> 1; h >= 1; h >>= 1) v = v + __shfl_down_sync(FULL, v, h);
    return __shfl_sync(FULL, v, 0);
}

// Integer sums are exact in any order.
__device__ int tree_sum(const int8_t *a, int nv, bool neg, int8_t *, int lane) {
    int v = 0;
    for (int i = lane; i < nv; i += 32) {
        const int x = a[i];
        v += neg ? (x < 0 ? -x : 0) : (x > 0 ? x : 0);
    }
    return __reduce_add_sync(FULL, v);
}

template <typename T>
__device__ __forceinline__ T *stage(T *alpha, int j) { return alpha + (1 << j); }

// F or G of a node of stage j starting at bit s: stage j (or the channel
// row when j = n) -> stage j - 1.
template <typename T, bool IS_G>
__device__ __forceinline__ void fg(const Sc1wParams &p, T *alpha, const uint32_t *bw, const T *ch, bool vec_ch,
                                   int j, int s, int lane) {
    typedef A1<T> A;
    const int h = 1 << (j - 1);
    const bool root = j == p.n;
    const T *in = root ? ch : stage(alpha, j);
    T *out = stage(alpha, j - 1);
    if (sizeof(T) == 1 && h >= 128 && (!root || vec_ch)) {
        const uint32_t *in4 = reinterpret_cast<const uint32_t *>(in);
        uint32_t *out4 = reinterpret_cast<uint32_t *>(out);
        const int h4 = h >> 2;
        for (int w = lane; w < h4; w += 32) {
            uint32_t a = root ? __ldg(in4 + w) : in4[w];
            uint32_t b = root ? __ldg(in4 + w + h4) : in4[w + h4];
            if (root) { a = __vmaxs4(a, 0x81818181u); b = __vmaxs4(b, 0x81818181u); }
            if (IS_G) {
                const int pos = s + 4 * w;
                out4[w] = g4(a, b, (bw[pos >> 5] >> (pos & 31)) & 0xFu);
            } else {
                out4[w] = f4(a, b);
            }
        }
        return;
    }
    if (sizeof(T) == 4 && h >= 128 && (!root || vec_ch)) {
        const float4 *in4 = reinterpret_cast<const float4 *>(in);
        float4 *out4 = reinterpret_cast<float4 *>(out);
        const int h4 = h >> 2;
        for (int w = lane; w < h4; w += 32) {
            const float4 a = root ? __ldg(in4 + w) : in4[w];
            const float4 b = root ? __ldg(in4 + w + h4) : in4[w + h4];
            float4 r;
            if (IS_G) {
                const int pos = s + 4 * w;
                const uint32_t nib = (bw[pos >> 5] >> (pos & 31)) & 0xFu;
                r.x = A1<float>::g(a.x, b.x, nib & 1u);
                r.y = A1<float>::g(a.y, b.y, (nib >> 1) & 1u);
                r.z = A1<float>::g(a.z, b.z, (nib >> 2) & 1u);
                r.w = A1<float>::g(a.w, b.w, (nib >> 3) & 1u);
            } else {
                r.x = A1<float>::f(a.x, b.x);
                r.y = A1<float>::f(a.y, b.y);
                r.z = A1<float>::f(a.z, b.z);
                r.w = A1<float>::f(a.w, b.w);
            }
            out4[w] = r;
        }
        return;
    }
    for (int e = lane; e < h; e += 32) {
        const typename A::V a = root ? A::ldch(in + e) : A::ld(in + e);
        const typename A::V b = root ? A::ldch(in + e + h) : A::ld(in + e + h);
        out[e] = A::st(IS_G ? A::g(a, b, beta_bit(bw, s + e)) : A::f(a, b));
    }
}

// Pairwise tree sum over lanes [base, base + nv) of t (zero elsewhere),
// returned to every lane: lane base + e adds lane base + e + h, h = nv/2, ...
template <typename V>
__device__ __forceinline__ V wsum(V t, int nv, int base) {
    for (int h = nv >> 1; h >= 1; h >>= 1) t = t + __shfl_down_sync(FULL, t, h);
    return __shfl_sync(FULL, t, base);
}

// A leaf of 64 or more bits, read from its stage in shared memory (a: its
// input, scr: the dead stage below it, scratch for float sums).
template <typename T>
__device__ void leaf_smem(int kind, const T *a, T *scr, uint32_t *bw, int nv, int s, typename A1<T>::V &pen,
                          int lane) {
    typedef A1<T> A;
    typedef typename A::V V;
    if (kind == OP_R0) {                                               // Eq. (10)
        pen = pen + tree_sum(a, nv, true, scr, lane);
        for (int c = 0; c < nv / 32; ++c) put_chunk(bw, s, nv, c, false, lane);
    } else if (kind == OP_R1) {
        for (int c = 0; c < nv / 32; ++c) put_chunk(bw, s, nv, c, A::ld(a + 32 * c + lane) < 0, lane);
    } else if (kind == OP_REP) {                                       // Eq. (5), ties to all zero
        const V p0 = tree_sum(a, nv, true, scr, lane);
        const V p1 = tree_sum(a, nv, false, scr, lane);
        const bool one = !(p0 <= p1);
        pen = pen + (one ? p1 : p0);
        for (int c = 0; c < nv / 32; ++c) put_chunk(bw, s, nv, c, one, lane);
    } else {                                                           // SPC, Sec. III-D
        uint32_t par = 0;
        unsigned long long best = ~0ull;
        for (int c = 0; c < nv / 32; ++c) {
            const int e = 32 * c + lane;
            const V x = A::ld(a + e);
            const unsigned long long key = ((unsigned long long)A::absbits(x) << 32) | (uint32_t)e;
            best = key < best ? key : best;
            par ^= (uint32_t)__popc(__ballot_sync(FULL, x < 0)) & 1u;
            put_chunk(bw, s, nv, c, x < 0, lane);
        }
        for (int off = 16; off >= 1; off >>= 1) {
            const unsigned long long o2 = __shfl_xor_sync(FULL, best, off);
            best = o2 < best ? o2 : best;
        }
        if (par) {
            const int e = (int)(uint32_t)best;
            __syncwarp();
            if (lane == 0) bw[(s + e) >> 5] ^= 1u << ((s + e) & 31);
            pen = pen + A::unabs((uint32_t)(best >> 32));
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kSc1wThreads, 6) sc1w_kernel(const Sc1wParams p) {
    typedef A1<T> A;
    typedef typename A::V V;                        // an LLR in arithmetic: float, or int for int8
    typedef V PT;                                   // penalty: float, or exact int for int8
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int N = 1 << p.n;
    const int bwn = N >= 32 ? N >> 5 : 1;
    uint8_t *mine = smem_raw + (size_t)warp * p.warp_bytes;
    T *alpha = reinterpret_cast<T *>(mine);
    uint32_t *bw = reinterpret_cast<uint32_t *>(mine + p.beta_off);
    const uint32_t count = p.frame_idx ? *p.frame_cnt : p.n_frames;
    const bool vec_ch = (reinterpret_cast<uintptr_t>(p.llr) & 15u) == 0;
    const uint32_t wpc = blockDim.x >> 5;
    for (uint32_t i = blockIdx.x * wpc + warp; i < count; i += gridDim.x * wpc) {
        const uint32_t f = p.frame_idx ? p.frame_idx[i] : i;
        const T *ch = reinterpret_cast<const T *>(p.llr) + (size_t)f * N;
        PT pen = 0;
        // The 32-bit window in registers: R holds alpha stages 0..4, stage j
        // in lanes [2^j, 2^(j+1)); R5 holds stage 5, element e in lane e; W
        // holds the window's 32 beta bits (lane 0 stores it after each change).
        V R = 0, R5 = 0;
        uint32_t W = 0;
        if (p.n <= 5) {
            if (p.n == 5) R5 = A::ldch(ch + lane);
            else if (lane >= N && lane < 2 * N) R = A::ldch(ch + lane - N);
        } else if (p.root_leaf) {
            T *top = stage(alpha, p.n);
            for (int e = lane; e < N; e += 32) top[e] = A::st(A::ldch(ch + e));
            __syncwarp();
        }
        // Only operations on shared memory synchronise the warp: the window
        // operations touch registers, and lane 0 alone stores W.
        uint32_t op = __ldg(p.ops);
        for (int o = 0; o < p.n_ops; ++o) {
            const uint32_t next = o + 1 < p.n_ops ? __ldg(p.ops + o + 1) : 0u;
            const int kind = (int)(op & 15u), j = (int)((op >> 4) & 15u), s = (int)(op >> 8);
            const int nv = 1 << j;
            if (kind == OP_F || kind == OP_G) {                        // Eq. (1), (2)
                const bool isg = kind == OP_G;
                if (j >= 7) {
                    __syncwarp();
                    if (isg) fg<T, true>(p, alpha, bw, ch, vec_ch, j, s, lane);
                    else fg<T, false>(p, alpha, bw, ch, vec_ch, j, s, lane);
                    __syncwarp();
                } else if (j == 6) {                                   // stage 6 -> R5
                    __syncwarp();
                    const bool root = p.n == 6;
                    const T *in = root ? ch : stage(alpha, 6);
                    const V a = root ? A::ldch(in + lane) : A::ld(in + lane);
                    const V b = root ? A::ldch(in + lane + 32) : A::ld(in + lane + 32);
                    R5 = isg ? A::g(a, b, (W >> lane) & 1u) : A::f(a, b);
                } else {                                               // inside the window
                    const int h = nv >> 1, e = lane & (h - 1);
                    const V src = j == 5 ? R5 : R;
                    const int base = j == 5 ? 0 : nv;
                    const V a = __shfl_sync(FULL, src, base + e);
                    const V b = __shfl_sync(FULL, src, base + e + h);
                    const V r = isg ? A::g(a, b, (W >> ((s & 31) + e)) & 1u) : A::f(a, b);
                    if (lane >= h && lane < nv) R = r;
                }
            } else if (kind == OP_COMB) {                              // Eq. (3), in place
                const int h = nv >> 1;
                if (h >= 32) {
                    __syncwarp();
                    for (int w = lane; w < (h >> 5); w += 32) bw[(s >> 5) + w] ^= bw[((s + h) >> 5) + w];
                    __syncwarp();
                } else {
                    W ^= (W >> h) & (((1u << h) - 1u) << (s & 31));
                    if (lane == 0) bw[s >> 5] = W;
                }
            } else if (j >= 6) {
                __syncwarp();
                leaf_smem<T>(kind, stage(alpha, j), stage(alpha, j - 1), bw, nv, s, pen, lane);
                __syncwarp();
            } else {                                                   // a leaf inside the window
                const V v = j == 5 ? R5 : R;
                const int base = j == 5 ? 0 : nv;
                const bool in = lane >= base && lane < base + nv;
                const uint32_t mask = j == 5 ? FULL : ((1u << nv) - 1u);
                uint32_t bits = 0;
                if (kind == OP_R0) {                                   // Eq. (10)
                    pen = pen + wsum<V>(in ? A::negpart(v) : V(0), nv, base);
                } else if (kind == OP_R1) {
                    bits = (__ballot_sync(FULL, in && v < 0) >> base) & mask;
                } else if (kind == OP_REP) {                           // Eq. (5), ties to all zero
                    const V p0 = wsum<V>(in ? A::negpart(v) : V(0), nv, base);
                    const V p1 = wsum<V>(in ? A::pospart(v) : V(0), nv, base);
                    const bool one = !(p0 <= p1);
                    pen = pen + (one ? p1 : p0);
                    bits = one ? mask : 0u;
                } else {                                               // SPC, Sec. III-D
                    bits = (__ballot_sync(FULL, in && v < 0) >> base) & mask;
                    unsigned long long key =
                        in ? (((unsigned long long)A::absbits(v) << 32) | (uint32_t)(lane - base)) : ~0ull;
                    for (int off = nv >> 1; off >= 1; off >>= 1) {
                        const unsigned long long o2 = __shfl_xor_sync(FULL, key, off);
                        key = o2 < key ? o2 : key;
                    }
                    key = __shfl_sync(FULL, key, base);
                    if (__popc(bits) & 1) {
                        bits ^= 1u << (uint32_t)key;
                        pen = pen + A::unabs((uint32_t)(key >> 32));
                    }
                }
                if (j == 5) {
                    W = bits;
                } else {
                    const int sh = s & 31;
                    W = (W & ~(mask << sh)) | (bits << sh);
                }
                if (lane == 0) bw[s >> 5] = W;
            }
            op = next;
        }
        __syncwarp();

        // ---------------- final pick (Sec. II-B) ----------------
        uint32_t acc = 0;
        if (p.crc_len > 0) {
            const uint8_t *xb = reinterpret_cast<const uint8_t *>(bw);
            for (int b = lane; b < (N >> 3); b += 32) acc ^= __ldg(p.syn + ((b << 8) | xb[b]));
            for (int off = 16; off >= 1; off >>= 1) acc ^= __shfl_xor_sync(FULL, acc, off);
        }
        __syncwarp();
        if (!p.systematic) {                                           // u = x G_N, in place
            const uint32_t M[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
            for (int w = lane; w < bwn; w += 32) {
                uint32_t u = bw[w];
#pragma unroll
                for (int e = 0; e < 5; ++e)
                    if ((1 << e) < N) u ^= (u >> (1 << e)) & M[e];
                bw[w] = u;
            }
            __syncwarp();
            for (int d = 1; d < bwn; d <<= 1) {
                for (int w = lane; w < bwn; w += 32)
                    if (!(w & d)) bw[w] ^= bw[w + d];
                __syncwarp();
            }
        }
        uint8_t *row = p.bits + (size_t)f * p.kb;
        for (int b = lane; b < p.kb; b += 32) {
            uint32_t byte = 0;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int pos = 8 * b + t;
                if (pos < p.k) {
                    const uint32_t u = __ldg(p.info + pos);
                    byte |= ((bw[u >> 5] >> (u & 31u)) & 1u) << t;
                }
            }
            row[b] = (uint8_t)byte;
        }
        if (lane == 0) {
            p.pm[f] = (float)pen;
            if (p.ok) p.ok[f] = (uint8_t)(p.crc_len == 0 || acc == 0u);
            if (p.slot) p.slot[f] = 0;
        }
        __syncwarp();
    }
}

}  // namespace

int sc1w_warp_bytes(int n, int es, bool root_leaf, int *beta_off) {
    const int N = 1 << n;
    const int a = ((root_leaf ? 2 * N : N) * es + 15) & ~15;
    const int b = ((N >= 32 ? N / 8 : 4) + 15) & ~15;
    if (beta_off) *beta_off = a;
    return a + b;
}

int occupancy_sc1w(int dtype, int n, bool root_leaf, int warps) {
    const int smem = warps * sc1w_warp_bytes(n, dtype == POLAR_LLR_I8 ? 1 : 4, root_leaf, nullptr);
    const void *fn = dtype == POLAR_LLR_I8 ? (const void *)sc1w_kernel<int8_t> : (const void *)sc1w_kernel<float>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, 32 * warps, smem) != cudaSuccess) return 0;
    return blocks;
}

cudaError_t launch_sc1w(int dtype, const Sc1wParams &p, int grid, int warps, cudaStream_t st) {
    const int smem = warps * p.warp_bytes;
    if (dtype == POLAR_LLR_I8) {
        cudaFuncSetAttribute(sc1w_kernel<int8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        sc1w_kernel<int8_t><<<grid, 32 * warps, smem, st>>>(p);
    } else {
        cudaFuncSetAttribute(sc1w_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        sc1w_kernel<float><<<grid, 32 * warps, smem, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace polar
