// polar_wide.cu -- list decoding with L = 64 or 128 paths.
//
// The narrow kernels (polar_kernels.cu) map one path to one lane of one warp.
// Wider lists (the paper uses L = 128 to study the CRC length, Sec. VI,
// Fig. 3) need more lanes than a warp has, so they run here: one CTA of L
// threads per frame, thread p owning path p for leaves, all threads sharing
// the element-wise F / G / Combine work. The schedule is the fully unrolled
// one (every F, G, Combine and leaf of the decoding tree, Sec. II-D,
// Listing 2); every stage lives in the CTA's global scratch (or, up to a
// shared-memory budget, the smallest buffers on chip) behind per-path
// stage-index rows (the lazy copy of Sec. IV-A/B). Selection (Algorithm 1)
// sorts all candidate keys of the CTA in shared memory and keeps the L
// smallest; survivors take slots in (source, candidate) order.
//
// The arithmetic is the narrow decoder's, element by element: min-sum F
// (Eq. (1)), G (Eq. (2), saturating for int8), Combine (Eq. (3)), the node
// rules of Sec. III-B..E with pairwise-tree sums, least reliable bits ranked
// by (|a|, index), penalties parent + increment, keys (penalty, source slot,
// candidate index), and the final CRC pick of Sec. II-B.

#include "polar_internal.h"

namespace polar {
namespace {

constexpr unsigned FULLW = 0xffffffffu;
constexpr unsigned long long KINF64 = ~0ull;

template <typename T> struct WA;
template <> struct WA<float> {
    typedef float P;
    static __device__ __forceinline__ float negp(float a) { return a < 0.f ? -a : 0.f; }
    static __device__ __forceinline__ float posp(float a) { return a > 0.f ? a : 0.f; }
    static __device__ __forceinline__ uint32_t absbits(float a) { return __float_as_uint(fabsf(a)); }
    static __device__ __forceinline__ float unabs(uint32_t b) { return __uint_as_float(b); }
    static __device__ __forceinline__ uint32_t pbits(float p) { return __float_as_uint(p); }
    static __device__ __forceinline__ float frombits(uint32_t b) { return __uint_as_float(b); }
    static __device__ __forceinline__ float f(float a, float b) {
        const float m = fminf(fabsf(a), fabsf(b));
        return __uint_as_float(__float_as_uint(m) | ((__float_as_uint(a) ^ __float_as_uint(b)) & 0x80000000u));
    }
    static __device__ __forceinline__ float g(float a, float b, uint32_t beta) {
        return b + __uint_as_float(__float_as_uint(a) ^ (beta << 31));
    }
};
template <> struct WA<int8_t> {
    typedef int P;
    static __device__ __forceinline__ int negp(int8_t a) { return a < 0 ? -(int)a : 0; }
    static __device__ __forceinline__ int posp(int8_t a) { return a > 0 ? (int)a : 0; }
    static __device__ __forceinline__ uint32_t absbits(int8_t a) { return (uint32_t)(a < 0 ? -(int)a : (int)a); }
    static __device__ __forceinline__ int unabs(uint32_t b) { return (int)b; }
    static __device__ __forceinline__ uint32_t pbits(int p) { return (uint32_t)p; }
    static __device__ __forceinline__ int frombits(uint32_t b) { return (int)b; }
    static __device__ __forceinline__ int8_t f(int8_t a, int8_t b) {
        const int x = a, y = b;
        const int m = min(abs(x), abs(y));
        return (int8_t)(((x ^ y) < 0) ? -m : m);
    }
    static __device__ __forceinline__ int8_t g(int8_t a, int8_t b, uint32_t beta) {
        const int r = beta ? (int)b - (int)a : (int)b + (int)a;
        return (int8_t)max(-127, min(127, r));
    }
};

__device__ __forceinline__ uint32_t spc_mask(int c) { return (0xFCA69530u >> (4 * c)) & 0xFu; }

// Four int8 LLRs in one word (lanes of the SIMD intrinsics): F of Eq. (1) as
// max(min(a, b), -max(a, b)), which is sign(a) sign(b) min(|a|, |b|) for
// values in [-127, 127]; G of Eq. (2) with the four beta bits in nib (bit e ->
// byte e), saturated to [-127, 127].
__device__ __forceinline__ uint32_t f4w(uint32_t a, uint32_t b) {
    return __vmaxs4(__vmins4(a, b), __vneg4(__vmaxs4(a, b)));
}
__device__ __forceinline__ uint32_t g4w(uint32_t a, uint32_t b, uint32_t nib) {
    const uint32_t m = ((nib * 0x00204081u) & 0x01010101u) * 0xFFu;   // byte e = 0xFF when bit e of nib
    const uint32_t sa = (a & ~m) | (__vneg4(a) & m);
    return __vmaxs4(__vaddss4(b, sa), 0x81818181u);
}

// Shared memory of one CTA (one frame at a time).
struct WideSmem {
    uint8_t *idx[2], *bidx[2];     // [L][16] stage -> physical row
    uint32_t *pen[2];              // penalty bits per slot
    unsigned long long *keys;      // [8][L] candidate keys, candidate-major: (source t, candidate c) at c * L + t,
                                   // so a warp's lanes touch consecutive words
    unsigned long long *sortb;     // [pow2 >= L * 8] sort buffer
    uint32_t *flag, *mpos;         // per source: SPC parity / repetition ML flag, [L][4] positions
    int *nsrc;                     // per new slot: index into keys[]
    int *scan;                     // [L] per-thread counts
    uint32_t *ubuf;                // winner's u words
    unsigned long long *red;       // [L / 32] reduction scratch
};

// Bytes of the CTA's tables (index rows, penalties, keys, sort buffer, ...), a multiple of 16.
__host__ __device__ __forceinline__ uint32_t tables_bytes(int L, int n) {
    const uint32_t b = (uint32_t)(4 * L * 16 + 2 * L * 4 + 2 * L * 8 * 8 + L * 4 + L * 16 + 2 * L * 4 +
                                  beta_words(n) * 4);
    return ((((b + 15u) & ~15u) + 8u * (uint32_t)(L / 32)) + 15u) & ~15u;
}

__device__ __forceinline__ WideSmem carve(uint8_t *base, int L, int nbw) {
    WideSmem s;
    uint8_t *p = base;
    for (int b = 0; b < 2; ++b) { s.idx[b] = p; p += L * 16; }
    for (int b = 0; b < 2; ++b) { s.bidx[b] = p; p += L * 16; }
    for (int b = 0; b < 2; ++b) { s.pen[b] = reinterpret_cast<uint32_t *>(p); p += L * 4; }
    s.keys = reinterpret_cast<unsigned long long *>(p); p += L * 8 * 8;
    s.sortb = reinterpret_cast<unsigned long long *>(p); p += L * 8 * 8;
    s.flag = reinterpret_cast<uint32_t *>(p); p += L * 4;
    s.mpos = reinterpret_cast<uint32_t *>(p); p += L * 16;
    s.nsrc = reinterpret_cast<int *>(p); p += L * 4;
    s.scan = reinterpret_cast<int *>(p); p += L * 4;
    s.ubuf = reinterpret_cast<uint32_t *>(p); p += nbw * 4;
    p = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
    s.red = reinterpret_cast<unsigned long long *>(p);
    return s;
}

// A buffer in the CTA's shared memory (SX: after its tables) or global scratch (G).
__device__ __forceinline__ uint8_t *wbuf(uint64_t loc, uint8_t *SX, uint8_t *G) {
    return (loc & kWideInSmem) ? SX + (uint32_t)loc : G + loc;
}

template <typename T>
__device__ __forceinline__ T *wrow(const WideView &v, uint8_t *SX, uint8_t *G, const WideSmem &s, int cur, int p,
                                   int j) {
    if (j == v.n) return reinterpret_cast<T *>(wbuf(v.gchan, SX, G));
    return reinterpret_cast<T *>(wbuf(v.galpha[j], SX, G)) + ((size_t)s.idx[cur][p * 16 + j] << j);
}

// CTA-wide exclusive scan of one int per thread; returns the prefix, *total the sum.
__device__ __forceinline__ int cta_excl_scan(int x, int *scan, int *total) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
    int v = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(FULLW, v, d);
        if (lane >= d) v += o;
    }
    if (lane == 31) scan[w] = v;
    __syncthreads();
    int base = 0, tot = 0;
    for (int i = 0; i < nw; ++i) {
        if (i < w) base += scan[i];
        tot += scan[i];
    }
    __syncthreads();
    *total = tot;
    return base + v - x;
}

// Compare-exchange across lanes at distance j (< 32): the lower lane of each
// pair keeps the smaller key when the run ascends, the larger one otherwise.
__device__ __forceinline__ unsigned long long ce_lanes(unsigned long long x, int lane, int j, bool up) {
    const unsigned long long y = __shfl_xor_sync(FULLW, x, j);
    const unsigned long long mn = x < y ? x : y, mx = x < y ? y : x;
    return (((lane & j) == 0) == up) ? mn : mx;
}

// Ascending bitonic sort of buf[0 .. P) by the CTA, P a power of two of at
// least 32: the network of the plain shared-memory sort, with every distance
// below 32 done by warp shuffles inside a 32-key chunk (warp w takes chunks w,
// w + warps, ... one at a time, one key per lane), so that only distances of
// 32 and more pass through shared memory with a CTA barrier after each.
__device__ void cta_sort(unsigned long long *buf, int P) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nch = P >> 5;
    for (int c = w; c < nch; c += nw) {
        unsigned long long x = buf[c * 32 + lane];
        for (int k = 2; k <= 32; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) x = ce_lanes(x, lane, j, ((c * 32 + lane) & k) == 0);
        buf[c * 32 + lane] = x;
    }
    __syncthreads();
    for (int k = 64; k <= P; k <<= 1) {
        for (int j = k >> 1; j >= 32; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int o = i ^ j;
                if (o > i) {
                    const unsigned long long a = buf[i], b = buf[o];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) { buf[i] = b; buf[o] = a; }
                }
            }
            __syncthreads();
        }
        for (int c = w; c < nch; c += nw) {
            unsigned long long x = buf[c * 32 + lane];
            const bool up = ((c * 32) & k) == 0;
#pragma unroll
            for (int j = 16; j > 0; j >>= 1) x = ce_lanes(x, lane, j, up);
            buf[c * 32 + lane] = x;
        }
        __syncthreads();
    }
}

// Exact L-th smallest of the M = La * C > L candidate keys, source t owning
// keys[c * L + t] for c < C. With a full list (La = L) the answer is at most t0, the
// largest of the sources' best keys, so only keys <= t0 are sorted: the L
// best keys plus the few later candidates below t0. Otherwise all M keys are.
__device__ __forceinline__ unsigned long long cta_kth(const WideSmem &s, int M, int L, int La, int C) {
    const int t = threadIdx.x;
    unsigned long long t0 = KINF64;
    if (La == L) {
        unsigned long long m = 0ull;
        if (t < La) {
            m = KINF64;
            for (int c = 0; c < C; ++c) m = s.keys[c * L + t] < m ? s.keys[c * L + t] : m;
        }
        for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(FULLW, m, d);
            m = o > m ? o : m;
        }
        if ((t & 31) == 0) s.red[t >> 5] = m;
        __syncthreads();
        t0 = s.red[0];
        for (int w = 1; w < ((int)blockDim.x >> 5); ++w) t0 = s.red[w] > t0 ? s.red[w] : t0;
        __syncthreads();
    }
    // compact the keys <= t0 (all of them without a full list)
    int cnt = 0;
    if (t < La)
        for (int c = 0; c < C; ++c) cnt += s.keys[c * L + t] <= t0 ? 1 : 0;
    int S = 0;
    int off = cta_excl_scan(cnt, s.scan, &S);
    if (S == L) return t0;               // no later candidate below t0
    if (t < La)
        for (int c = 0; c < C; ++c)
            if (s.keys[c * L + t] <= t0) s.sortb[off++] = s.keys[c * L + t];
    int P = 32;
    while (P < S) P <<= 1;
    for (int i = S + t; i < P; i += blockDim.x) s.sortb[i] = KINF64;
    __syncthreads();
    cta_sort(s.sortb, P);
    return s.sortb[L - 1];
}

// Canonical sums of |min(a,0)| and |max(a,0)| over nv elements (in place on
// the path's own row, which the leaf does not need afterwards).
template <typename T>
__device__ __forceinline__ void wide_sums(T *row, int nv, bool want1, typename WA<T>::P &v0, typename WA<T>::P &v1) {
    typedef typename WA<T>::P P;
    if (sizeof(T) == 1) {
        int s0 = 0, s1 = 0;
        for (int i = 0; i < nv; ++i) {
            s0 += WA<T>::negp(row[i]);
            s1 += WA<T>::posp(row[i]);
        }
        v0 = (P)s0;
        v1 = (P)s1;
        return;
    }
    float *x = reinterpret_cast<float *>(row);
    if (nv == 1) {
        v0 = (P)WA<float>::negp(x[0]);
        v1 = (P)WA<float>::posp(x[0]);
        return;
    }
    const int h = nv >> 1;
    for (int i = 0; i < h; ++i) {
        const float a = x[i], b = x[i + h];
        x[i] = WA<float>::negp(a) + WA<float>::negp(b);
        x[i + h] = WA<float>::posp(a) + WA<float>::posp(b);
    }
    for (int hh = h >> 1; hh >= 1; hh >>= 1) {
        for (int i = 0; i < hh; ++i) {
            x[i] = x[i] + x[i + hh];
            x[h + i] = x[h + i] + x[h + i + hh];
        }
    }
    v0 = (P)x[0];
    v1 = want1 ? (P)x[h] : (P)0;
}

template <typename T>
__device__ void wide_frame(const WideView &v, uint8_t *SX, uint8_t *G, const WideSmem &s, const uint8_t *src,
                           uint8_t *bits_row,
                           float *pm_out, uint8_t *ok_out, int32_t *slot_out) {
    typedef typename WA<T>::P P;
    const int t = threadIdx.x, nt = blockDim.x, lane = t & 31;
    const int n = v.n, N = v.N, L = v.L;
    const int nbw = beta_words(n);
    T *chan = reinterpret_cast<T *>(wbuf(v.gchan, SX, G));
    uint32_t *br = reinterpret_cast<uint32_t *>(wbuf(v.gbr, SX, G));

    for (int i = t; i < N; i += nt) {
        T x = reinterpret_cast<const T *>(src)[i];
        if (sizeof(T) == 1 && (int)x < -127) x = (T)-127;   // -128 reads as -127
        chan[i] = x;
    }
    for (int i = t; i < L * 16; i += nt) {
        s.idx[0][i] = 0; s.idx[1][i] = 0; s.bidx[0][i] = 0; s.bidx[1][i] = 0;
    }
    if (t == 0) s.pen[0][0] = 0u;
    __syncthreads();
    int La = 1, cur = 0;

    for (int o = 0; o < v.n_xops; ++o) {
        const uint32_t op = __ldg(v.xops + o);
        const uint32_t kind = op_kind(op);
        const int j = op_stage(op);
        const int dest = op_dest(op);
        if (kind == OP_F || kind == OP_G) {
            const int jo = j - 1, h = 1 << jo;
            const int bwc = beta_words(jo);
            const uint32_t *blb = reinterpret_cast<const uint32_t *>(wbuf(v.gbl[jo], SX, G));
            T *outb = reinterpret_cast<T *>(wbuf(v.galpha[jo], SX, G));
            // L = 128: several 16-byte items in flight per thread; L = 64 (64
            // threads) measured faster with one 4-element item per pass
            if (L >= 128 && sizeof(T) == 4 && h >= 4) {
                // float4 items, four in flight per thread
                const int lq = jo - 2;
                const int total = La << lq;
                for (int e0 = t; e0 < total; e0 += 4 * nt) {
                    float4 a[4], b[4];
                    uint32_t nb[4] = {0u, 0u, 0u, 0u};
                    int pp[4], ii[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int e = e0 + u * nt;
                        pp[u] = e < total ? e >> lq : 0;
                        ii[u] = e < total ? (e & ((h >> 2) - 1)) << 2 : 0;
                        const float *in = reinterpret_cast<const float *>(wrow<T>(v, SX, G, s, cur, pp[u], j));
                        a[u] = *reinterpret_cast<const float4 *>(in + ii[u]);
                        b[u] = *reinterpret_cast<const float4 *>(in + ii[u] + h);
                        if (kind == OP_G)
                            nb[u] = (blb[(int)s.bidx[cur][pp[u] * 16 + jo] * bwc + (ii[u] >> 5)] >> (ii[u] & 31)) & 15u;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (e0 + u * nt >= total) break;
                        float4 r;
                        if (kind == OP_F) {
                            r.x = WA<float>::f(a[u].x, b[u].x); r.y = WA<float>::f(a[u].y, b[u].y);
                            r.z = WA<float>::f(a[u].z, b[u].z); r.w = WA<float>::f(a[u].w, b[u].w);
                        } else {
                            r.x = WA<float>::g(a[u].x, b[u].x, nb[u] & 1u);
                            r.y = WA<float>::g(a[u].y, b[u].y, (nb[u] >> 1) & 1u);
                            r.z = WA<float>::g(a[u].z, b[u].z, (nb[u] >> 2) & 1u);
                            r.w = WA<float>::g(a[u].w, b[u].w, (nb[u] >> 3) & 1u);
                        }
                        *reinterpret_cast<float4 *>(reinterpret_cast<float *>(outb) + ((size_t)pp[u] << jo) + ii[u]) = r;
                    }
                }
            } else if (L >= 128 && sizeof(T) == 1 && h >= 16) {
                // 16-byte items of int8 LLRs (four-lane SIMD words), two in flight per thread
                const int lq = jo - 4;
                const int total = La << lq;
                for (int e0 = t; e0 < total; e0 += 2 * nt) {
                    uint4 a[2], b[2];
                    uint32_t nb[2] = {0u, 0u};
                    int pp[2], ii[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int e = e0 + u * nt;
                        pp[u] = e < total ? e >> lq : 0;
                        ii[u] = e < total ? (e & ((h >> 4) - 1)) << 4 : 0;
                        const int8_t *in = reinterpret_cast<const int8_t *>(wrow<T>(v, SX, G, s, cur, pp[u], j));
                        a[u] = *reinterpret_cast<const uint4 *>(in + ii[u]);
                        b[u] = *reinterpret_cast<const uint4 *>(in + ii[u] + h);
                        if (kind == OP_G)
                            nb[u] = (blb[(int)s.bidx[cur][pp[u] * 16 + jo] * bwc + (ii[u] >> 5)] >> (ii[u] & 31)) & 0xFFFFu;
                    }
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (e0 + u * nt >= total) break;
                        uint4 r;
                        if (kind == OP_F) {
                            r.x = f4w(a[u].x, b[u].x); r.y = f4w(a[u].y, b[u].y);
                            r.z = f4w(a[u].z, b[u].z); r.w = f4w(a[u].w, b[u].w);
                        } else {
                            r.x = g4w(a[u].x, b[u].x, nb[u] & 15u); r.y = g4w(a[u].y, b[u].y, (nb[u] >> 4) & 15u);
                            r.z = g4w(a[u].z, b[u].z, (nb[u] >> 8) & 15u); r.w = g4w(a[u].w, b[u].w, (nb[u] >> 12) & 15u);
                        }
                        *reinterpret_cast<uint4 *>(reinterpret_cast<int8_t *>(outb) + ((size_t)pp[u] << jo) + ii[u]) = r;
                    }
                }
            } else if (h >= 4) {
                // four consecutive elements per item (16-byte float / 4-byte int8 vectors)
                const int lq = jo - 2;
                for (int e = t; e < (La << lq); e += nt) {
                    const int p = e >> lq, i = (e & ((h >> 2) - 1)) << 2;
                    const T *in = wrow<T>(v, SX, G, s, cur, p, j);
                    uint32_t bits4 = 0u;
                    if (kind == OP_G)
                        bits4 = (blb[(int)s.bidx[cur][p * 16 + jo] * bwc + (i >> 5)] >> (i & 31)) & 15u;
                    T x[4], y[4], r[4];
                    if (sizeof(T) == 4) {
                        const float4 a = *reinterpret_cast<const float4 *>(in + i);
                        const float4 b = *reinterpret_cast<const float4 *>(in + i + h);
                        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
                        for (int q = 0; q < 4; ++q) { x[q] = (T)av[q]; y[q] = (T)bv[q]; }
                    } else {
                        const uint32_t a = *reinterpret_cast<const uint32_t *>(in + i);
                        const uint32_t b = *reinterpret_cast<const uint32_t *>(in + i + h);
                        for (int q = 0; q < 4; ++q) {
                            x[q] = (T)(int8_t)((a >> (8 * q)) & 0xFF);
                            y[q] = (T)(int8_t)((b >> (8 * q)) & 0xFF);
                        }
                    }
                    for (int q = 0; q < 4; ++q)
                        r[q] = kind == OP_F ? WA<T>::f(x[q], y[q]) : WA<T>::g(x[q], y[q], (bits4 >> q) & 1u);
                    T *o = outb + ((size_t)p << jo) + i;
                    if (sizeof(T) == 4) {
                        *reinterpret_cast<float4 *>(o) = make_float4((float)r[0], (float)r[1], (float)r[2], (float)r[3]);
                    } else {
                        *reinterpret_cast<uint32_t *>(o) = ((uint32_t)(uint8_t)r[0]) | ((uint32_t)(uint8_t)r[1] << 8) |
                                                           ((uint32_t)(uint8_t)r[2] << 16) |
                                                           ((uint32_t)(uint8_t)r[3] << 24);
                    }
                }
            } else {
                for (int e = t; e < (La << jo); e += nt) {
                    const int p = e >> jo, i = e & (h - 1);
                    const T *in = wrow<T>(v, SX, G, s, cur, p, j);
                    T r;
                    if (kind == OP_F) {
                        r = WA<T>::f(in[i], in[i + h]);
                    } else {
                        const uint32_t bit = (blb[(int)s.bidx[cur][p * 16 + jo] * bwc + (i >> 5)] >> (i & 31)) & 1u;
                        r = WA<T>::g(in[i], in[i + h], bit);
                    }
                    outb[((size_t)p << jo) + i] = r;
                }
            }
            // this op reads only the stage-j entries of the index rows
            if (t < La) s.idx[cur][t * 16 + jo] = (uint8_t)t;
            __syncthreads();
        } else if (kind == OP_COMB) {
            const int jc = j - 1, bwc = beta_words(jc);
            const uint32_t *blb = reinterpret_cast<const uint32_t *>(wbuf(v.gbl[jc], SX, G));
            uint32_t *out = dest ? br : reinterpret_cast<uint32_t *>(wbuf(v.gbl[j], SX, G));
            const int ostride = dest ? nbw : beta_words(j);
            if (jc >= 5) {
                for (int e = t; e < La * bwc; e += nt) {
                    const int p = e / bwc, w = e - p * bwc;
                    const uint32_t l = blb[(int)s.bidx[cur][p * 16 + jc] * bwc + w];
                    const uint32_t r = br[p * nbw + w];
                    out[p * ostride + w] = l ^ r;
                    out[p * ostride + w + bwc] = r;
                }
            } else {
                const int hb = 1 << jc;
                const uint32_t m = (1u << hb) - 1u;
                if (t < La) {
                    const uint32_t l = blb[(int)s.bidx[cur][t * 16 + jc]];
                    const uint32_t r = br[t * nbw];
                    out[t * ostride] = ((l ^ r) & m) | ((r & m) << hb);
                }
            }
            // this op reads only the stage-jc entries of the left-beta rows
            if (!dest && t < La) s.bidx[cur][t * 16 + j] = (uint8_t)t;
            __syncthreads();
        } else {
            // ---------------- leaf of 2^j bits: thread p = path p ----------------
            const int nv = 1 << j;
            const int bw = beta_words(j);
            uint32_t *bout = dest ? br : reinterpret_cast<uint32_t *>(wbuf(v.gbl[j], SX, G));
            const int ostride = dest ? nbw : bw;
            const uint32_t wmask = nv >= 32 ? 0xffffffffu : ((1u << nv) - 1u);
            const bool act = t < La;
            if (kind == OP_R0) {
                // Rate-0 (Sec. III-B): penalty += sum |min(a, 0)|, beta = 0, no fork.
                if (act) {
                    T *row = wrow<T>(v, SX, G, s, cur, t, j);
                    P v0, v1;
                    wide_sums<T>(row, nv, false, v0, v1);
                    s.pen[cur][t] = WA<T>::pbits(WA<T>::frombits(s.pen[cur][t]) + v0);
                    for (int w = 0; w < bw; ++w) bout[t * ostride + w] = 0u;
                    if (!dest) s.bidx[cur][t * 16 + j] = (uint8_t)t;
                }
                __syncthreads();
                continue;
            }
            int C = 2;
            if (kind == OP_R1) C = nv == 1 ? 2 : 4;
            else if (kind == OP_SPC) C = L == 2 ? 2 : 8;
            if (act) {
                T *row = wrow<T>(v, SX, G, s, cur, t, j);
                const P ps = WA<T>::frombits(s.pen[cur][t]);
                unsigned long long *kk = s.keys + t;        // candidate c at kk[c * L]
                if (kind == OP_REP) {
                    // Repetition (Sec. III-E): the ML word listed first.
                    P x0, x1;
                    wide_sums<T>(row, nv, true, x0, x1);
                    const uint32_t fl = (x0 <= x1) ? 0u : 1u;
                    s.flag[t] = fl;
                    kk[0] = ((unsigned long long)WA<T>::pbits(ps + (fl ? x1 : x0)) << 32) | (unsigned)(t * C);
                    kk[L] = ((unsigned long long)WA<T>::pbits(ps + (fl ? x0 : x1)) << 32) | (unsigned)(t * C + 1);
                } else {
                    // least reliable positions by (|a|, index), and the parity of the hard decision
                    const int R = kind == OP_R1 ? 2 : 4;
                    unsigned long long top[4] = {KINF64, KINF64, KINF64, KINF64};
                    int neg = 0;
                    for (int i0 = 0; i0 < nv; i0 += 4) {
                        T q[4];
                        const int nq = nv < 4 ? nv : 4;
                        if (nv >= 4 && sizeof(T) == 4) {
                            const float4 f = *reinterpret_cast<const float4 *>(row + i0);
                            q[0] = (T)f.x; q[1] = (T)f.y; q[2] = (T)f.z; q[3] = (T)f.w;
                        } else if (nv >= 4) {
                            const uint32_t w = *reinterpret_cast<const uint32_t *>(row + i0);
                            for (int e = 0; e < 4; ++e) q[e] = (T)(int8_t)((w >> (8 * e)) & 0xFF);
                        } else {
                            for (int e = 0; e < nq; ++e) q[e] = row[i0 + e];
                        }
                        for (int e = 0; e < nq; ++e) {
                            const T a = q[e];
                            neg += a < (T)0 ? 1 : 0;
                            unsigned long long key = ((unsigned long long)WA<T>::absbits(a) << 16) | (unsigned)(i0 + e);
                            if (key < top[R - 1]) {
                                for (int r = 0; r < R; ++r)
                                    if (key < top[r]) { const unsigned long long x = top[r]; top[r] = key; key = x; }
                            }
                        }
                    }
                    P ar[4];
                    for (int r = 0; r < 4; ++r) {
                        ar[r] = WA<T>::unabs((uint32_t)(top[r] >> 16));
                        s.mpos[t * 4 + r] = (uint32_t)(top[r] & 0xFFFFu);
                    }
                    if (kind == OP_R1) {
                        // Rate-1 (Sec. III-C): HD, HD^m1, HD^m2, HD^m1^m2.
                        kk[0] = ((unsigned long long)WA<T>::pbits(ps) << 32) | (unsigned)(t * C);
                        kk[L] = ((unsigned long long)WA<T>::pbits(ps + ar[0]) << 32) | (unsigned)(t * C + 1);
                        if (C == 4) {
                            kk[2 * L] = ((unsigned long long)WA<T>::pbits(ps + ar[1]) << 32) | (unsigned)(t * C + 2);
                            kk[3 * L] = ((unsigned long long)WA<T>::pbits(ps + (ar[0] + ar[1])) << 32) | (unsigned)(t * C + 3);
                        }
                    } else {
                        // SPC (Sec. III-D): ML = HD or HD^m1 by the parity q; ML ^ T, penalty Eq. (9).
                        const uint32_t fl = (neg & 1) ? 0u : 1u;
                        s.flag[t] = fl;
                        for (int c = 0; c < C; ++c) {
                            const uint32_t dm = spc_mask(c) ^ (fl ? 0u : 1u);
                            P inc = (P)0;
                            bool first = true;
                            for (int r = 0; r < 4; ++r)
                                if ((dm >> r) & 1u) { inc = first ? ar[r] : inc + ar[r]; first = false; }
                            kk[c * L] = ((unsigned long long)WA<T>::pbits(ps + inc) << 32) | (unsigned)(t * C + c);
                        }
                    }
                }
            }
            __syncthreads();
            // ---------------- selection (Algorithm 1) ----------------
            const int M = La * C;
            const int keep = M < L ? M : L;
            const unsigned long long tau = M > L ? cta_kth(s, M, L, La, C) : KINF64;
            // survivors in (source, candidate) order: thread t scans items [t*q, t*q + q)
            const int q = (M + nt - 1) / nt;
            int cnt = 0;
            for (int i = t * q; i < M && i < t * q + q; ++i) cnt += s.keys[(i & (C - 1)) * L + i / C] <= tau ? 1 : 0;
            int tot = 0;
            int off = cta_excl_scan(cnt, s.scan, &tot);
            for (int i = t * q; i < M && i < t * q + q; ++i)
                if (s.keys[(i & (C - 1)) * L + i / C] <= tau) s.nsrc[off++] = i;
            __syncthreads();
            // ---------------- commit: slot t takes its source's rows and its word ----------------
            const int nxt = cur ^ 1;
            if (t < keep) {
                const int ki = s.nsrc[t];
                const int sp = ki / C, c = ki - sp * C;
                const unsigned long long key = s.keys[(ki & (C - 1)) * L + ki / C];
                s.pen[nxt][t] = (uint32_t)(key >> 32);
                reinterpret_cast<uint4 *>(s.idx[nxt])[t] = reinterpret_cast<const uint4 *>(s.idx[cur])[sp];
                reinterpret_cast<uint4 *>(s.bidx[nxt])[t] = reinterpret_cast<const uint4 *>(s.bidx[cur])[sp];
                if (!dest) s.bidx[nxt][t * 16 + j] = (uint8_t)t;
                uint32_t *ob = bout + t * ostride;
                if (kind == OP_REP) {
                    const uint32_t word = ((s.flag[sp] != 0u) != (c == 1)) ? wmask : 0u;
                    for (int w = 0; w < bw; ++w) ob[w] = word;
                } else {
                    const uint32_t dm = kind == OP_R1 ? (uint32_t)c : (spc_mask(c) ^ (s.flag[sp] ? 0u : 1u));
                    const T *srow = wrow<T>(v, SX, G, s, cur, sp, j);
                    for (int w = 0; w < bw; ++w) {
                        uint32_t word = 0;
                        const int lim = nv < 32 ? nv : 32;
                        if (lim >= 4 && sizeof(T) == 4) {
                            for (int i = 0; i < lim; i += 4) {
                                const float4 f = *reinterpret_cast<const float4 *>(srow + 32 * w + i);
                                word |= ((f.x < 0.f ? 1u : 0u) | (f.y < 0.f ? 2u : 0u) | (f.z < 0.f ? 4u : 0u) |
                                         (f.w < 0.f ? 8u : 0u)) << i;
                            }
                        } else if (lim >= 4) {
                            for (int i = 0; i < lim; i += 4) {
                                const uint32_t x = *reinterpret_cast<const uint32_t *>(srow + 32 * w + i);
                                const uint32_t sg = (x >> 7) & 0x01010101u;     // sign bit of each byte
                                word |= (((sg * 0x01020408u) >> 24) & 0xFu) << i;
                            }
                        } else {
                            for (int i = 0; i < lim; ++i) word |= (srow[32 * w + i] < (T)0 ? 1u : 0u) << i;
                        }
                        for (int r = 0; r < 4; ++r) {
                            const uint32_t m = s.mpos[sp * 4 + r];
                            if (((dm >> r) & 1u) && (int)(m >> 5) == w) word ^= 1u << (m & 31u);
                        }
                        ob[w] = word;
                    }
                }
            }
            __syncthreads();
            La = keep;
            cur = nxt;
        }
    }

    // ---------------- final pick (Sec. II-B) ----------------
    unsigned long long key = KINF64;
    if (t < La) {
        uint32_t acc = 0;
        if (v.crc_len > 0) {
            const uint8_t *xb = reinterpret_cast<const uint8_t *>(br + t * nbw);
            for (int b = 0; b < (N >> 3); ++b) acc ^= __ldg(v.syn + ((b << 8) | xb[b]));
        }
        key = ((unsigned long long)(acc != 0u ? 1u : 0u) << 63) | ((unsigned long long)s.pen[cur][t] << 8) |
              (unsigned long long)t;
    }
    for (int m = 16; m >= 1; m >>= 1) {
        const unsigned long long o2 = __shfl_xor_sync(FULLW, key, m);
        key = o2 < key ? o2 : key;
    }
    if (lane == 0) s.red[t >> 5] = key;
    __syncthreads();
    key = s.red[0];
    for (int w = 1; w < (nt >> 5); ++w) key = s.red[w] < key ? s.red[w] : key;
    const int win = (int)(key & 0xFFu);
    if (t < 32) {
        // u = x G_N for the winner (natural-order butterflies); a systematic code keeps x
        const uint32_t *xw = br + win * nbw;
        const int R = nbw > 32 ? nbw >> 5 : 1;
        uint32_t U[4];
        for (int r = 0; r < 4; ++r) {
            const int w = lane + 32 * r;
            U[r] = (r < R && w < nbw) ? xw[w] : 0u;
        }
        if (!v.systematic) {
            const uint32_t Mk[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
            for (int r = 0; r < 4; ++r)
                for (int e = 0; e < 5; ++e)
                    if ((1 << e) < N) U[r] ^= (U[r] >> (1 << e)) & Mk[e];
            for (int d = 1; d < nbw; d <<= 1) {
                if (d >= 32) {
                    const int dr = d >> 5;
                    for (int r = 0; r < 4; ++r)
                        if (r < R && !(r & dr) && r + dr < 4) U[r] ^= U[r + dr];
                } else {
                    for (int r = 0; r < 4; ++r) {
                        const uint32_t x = __shfl_down_sync(FULLW, U[r], d);
                        if (!(lane & d)) U[r] ^= x;
                    }
                }
            }
        }
        for (int r = 0; r < 4; ++r) {
            const int w = lane + 32 * r;
            if (r < R && w < nbw) s.ubuf[w] = U[r];
        }
        if (t == 0) {
            *pm_out = (float)WA<T>::frombits(s.pen[cur][win]);
            if (ok_out) *ok_out = (uint8_t)((key >> 63) ^ 1ull);
            if (slot_out) *slot_out = win;
        }
    }
    __syncthreads();
    for (int b = t; b < v.kb; b += nt) {
        uint32_t byte = 0;
        for (int e = 0; e < 8; ++e) {
            const int pos = 8 * b + e;
            if (pos < v.k) {
                const uint32_t u = __ldg(v.info + pos);
                byte |= ((s.ubuf[u >> 5] >> (u & 31u)) & 1u) << e;
            }
        }
        bits_row[b] = (uint8_t)byte;
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(128) wide_kernel(const WideParams P) {
    extern __shared__ __align__(16) uint8_t smem_w[];
    const WideView &v = P.v;
    const WideSmem s = carve(smem_w, v.L, beta_words(v.n));
    uint8_t *SX = smem_w + tables_bytes(v.L, v.n);
    uint8_t *G = P.scratch ? P.scratch + (size_t)blockIdx.x * v.gbytes : nullptr;
    const size_t nbytes = (size_t)v.N * sizeof(T);
    const uint32_t nf = P.frame_idx ? *P.frame_cnt : P.n_frames;
    for (uint32_t i = blockIdx.x; i < nf; i += gridDim.x) {
        const uint32_t f = P.frame_idx ? P.frame_idx[i] : i;
        wide_frame<T>(v, SX, G, s, reinterpret_cast<const uint8_t *>(P.llr) + (size_t)f * nbytes,
                      P.bits + (size_t)f * v.kb, P.pm + f, P.ok ? P.ok + f : nullptr, P.slot ? P.slot + f : nullptr);
    }
}

}  // namespace

uint32_t wide_smem_bytes(int L, int n) { return tables_bytes(L, n); }

int occupancy_wide(int dtype, int L, uint32_t sm) {
    int nb = 0;
    const void *fn = dtype == 0 ? (const void *)wide_kernel<float> : (const void *)wide_kernel<int8_t>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess) return 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, L, sm);
    return e == cudaSuccess ? nb : 0;
}

cudaError_t launch_wide(int dtype, const WideParams &p, int grid, cudaStream_t st) {
    const uint32_t sm = wide_smem_bytes(p.v.L, p.v.n) + p.v.sbytes;
    if (dtype == 0) {
        cudaFuncSetAttribute(wide_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        wide_kernel<float><<<grid, p.v.L, sm, st>>>(p);
    } else {
        cudaFuncSetAttribute(wide_kernel<int8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        wide_kernel<int8_t><<<grid, p.v.L, sm, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace polar
