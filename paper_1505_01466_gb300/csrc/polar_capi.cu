// polar_capi.cu -- host side of the C ABI declared in include/polar.h.
//
// polar_code_create turns a code description into what the decode kernels
// run: the Fast-SSC decoding tree flattened into an unrolled operation list
// (Sec. II-D, Listing 2) with small subtrees collapsed into register
// operations, the information positions, the CRC syndrome tables and a
// launch shape (warps per frame, CTA size, which alpha stages sit in shared
// memory and which spill to global scratch). The rest of the file drives the
// kernels: the plain, host-buffer, allocation-free and adaptive (Sec. V)
// decodes, the autotuner, wide lists (L = 64, 128), the batched form (work
// plan, persistent launch, CUDA graph) and the serving engine (admission by
// device memory, continuous batching on a host thread).

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/polar.h"
#include "polar_internal.h"

using namespace polar;

// Shared memory a wide-list CTA gives its smallest buffers by default: none.
// Measured at (1024, k=828) L = 128, every byte moved on chip costs more in
// CTAs per SM than it saves (0.34 M frames/s with none, 0.23 M with 48 KB).
constexpr uint32_t kWideDefaultBudget = 0u;
// Codes with at most this many paths pack their register subtrees (several
// frames to a warp, selection in L-lane segments) unless told otherwise:
// measured faster at L = 2 and 4 and slower at L = 8 and 16, where a frame's
// lane-per-path code on its own warp wins.
constexpr uint32_t kPackDefaultMaxL = 4u;

struct polar_code {
    uint32_t N, n, K, k, L, crc_len, flags;
    uint64_t crc_poly;
    std::vector<uint8_t> frozen;
    std::vector<uint32_t> ops;          // device schedule (small subtrees as OP_SUB)
    std::vector<uint32_t> xops;         // fully unrolled schedule (one entry per F/G/Combine/leaf)
    std::vector<unsigned long long> desc;  // subtree descriptors, two words each
    std::vector<int32_t> sched;         // (kind, N_v, start) triples of xops
    std::vector<uint16_t> info;         // information positions
    std::vector<uint32_t> syn;          // [N/8][256]
    uint32_t n_leaves = 0, n_r0 = 0, n_r1 = 0, n_rep = 0, n_spc = 0;
    bool host_only = false;
    int device = -1;
    int sm_count = 0;
    std::vector<uint32_t> shape_ops[2];  // ops with solo / sync flags of shape[d]
    uint32_t *d_syn = nullptr;
    uint16_t *d_info = nullptr;
    unsigned long long *d_desc = nullptr;
    LaunchShape shape[2];
    // Latency shape for small batches (at most one frame per SM): 4 warps per
    // frame, as much shared memory as a CTA has. Used unless set_launch fixed
    // the shape.
    LaunchShape lat[2];
    bool explicit_shape[2] = {false, false};
    // L = 64 / 128: the wide kernel over the fully unrolled schedule
    bool wide = false;
    uint32_t *d_xops = nullptr;
    uint32_t wide_budget[2] = {kWideDefaultBudget, kWideDefaultBudget};   // shared memory for its buffers
    // L = 1: the Fast-SSC kernel over sc1_op entries (used unless set_launch
    // fixed a shape of the list kernels)
    std::vector<uint32_t> sops;
    uint32_t *d_sops = nullptr;
    // shared memory per warp (32 frames) the L = 1 kernel may use; the
    // largest alpha stages above it go to global scratch
    uint32_t sc1_budget[2] = {0, 0};
    // Top alpha stages that may be evaluated from the channel instead of
    // stored (every node there an inner node of the list schedule, at most
    // three stages, none below stage kSubLog + 2), and the number in use for
    // each LLR type.
    uint32_t vmax = 0;
    uint32_t vdepth[2] = {0, 0};
    // Pack register subtrees (L <= 16) wherever the launch shape allows it
    // (one warp per frame), per LLR type: the plain, batched and serving forms
    // follow it; set_packing and the autotuner change it.
    bool pack_pref[2] = {false, false};
};

// Whether a shape of `warps` warps per frame runs the packed design.
bool packs(const polar_code *c, int dtype, uint32_t warps) {
    return warps == 1 && c->L <= 16 && c->pack_pref[dtype];
}

namespace {

// ---- test hooks (polar_debug_inject): host-side faults, no device fault ------
std::atomic<int64_t> g_fail_alloc_after{-1};   // < 0: off; else allocations left before failing
std::atomic<int> g_poison{0};

// Device allocation of a decode call; fails on purpose when the hook says so.
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t st, bool async = true) {
    int64_t k = g_fail_alloc_after.load();
    while (k >= 0) {
        if (k == 0) return cudaErrorMemoryAllocation;
        if (g_fail_alloc_after.compare_exchange_weak(k, k - 1)) break;
    }
    return async ? cudaMallocAsync(p, bytes, st) : cudaMalloc(p, bytes);
}

// Fill scratch with bytes no decode writes before reading (float NaN, int8 -128).
void scratch_poison(void *p, size_t bytes, int dtype, cudaStream_t st) {
    if (p && bytes && g_poison.load()) cudaMemsetAsync(p, dtype == POLAR_LLR_F32 ? 0xFF : 0x80, bytes, st);
}

// ---- launches from several host threads ------------------------------------
// The kernels' launch helpers raise the function's dynamic shared-memory limit
// to what the launch needs just before launching it (and the occupancy queries
// do the same). The limit belongs to the function, not to the call, so two
// threads launching the same kernel with different sizes could lower it in
// between; these wrappers make each set-and-launch (or set-and-query) atomic.
std::mutex g_launch_mu;

int occupancy_locked(int dtype, const LaunchShape &sh) {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    return occupancy(dtype, sh);
}
cudaError_t launch_decode_locked(int dtype, const LaunchShape &sh, const Params &p, int grid, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    return launch_decode(dtype, sh, p, grid, st);
}
int occupancy_batch_locked(int dtype, int warps, bool seg, uint32_t smem, int threads) {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    return occupancy_batch(dtype, warps, seg, smem, threads);
}
cudaError_t launch_batch_locked(int dtype, int warps, bool seg, const BatchParams &b, int grid, uint32_t smem,
                                int threads, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    return launch_batch(dtype, warps, seg, b, grid, smem, threads, st);
}
int occupancy_sc1_locked(int dtype, uint32_t warp_bytes, int warps, bool drop) {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    return occupancy_sc1(dtype, warp_bytes, warps, drop);
}
cudaError_t launch_sc1_locked(int dtype, const Sc1Params &p, int grid, int warps, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    return launch_sc1(dtype, p, grid, warps, st);
}
int occupancy_sc1w_locked(int dtype, int n, bool root_leaf, int warps) {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    return occupancy_sc1w(dtype, n, root_leaf, warps);
}
cudaError_t launch_sc1w_locked(int dtype, const Sc1wParams &p, int grid, int warps, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    return launch_sc1w(dtype, p, grid, warps, st);
}

// NVTX range for the duration of a host call (visible in Nsight timelines).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

uint32_t al16(uint32_t x) { return (x + 15u) & ~15u; }
uint64_t al256(uint64_t x) { return (x + 255u) & ~uint64_t(255); }

// ---- decoding tree (Sec. II-D) ----------------------------------------------
// Top down, first match wins: all frozen -> Rate-0; none frozen -> Rate-1;
// only the last bit information (N_v >= 2) -> repetition; only the first bit
// frozen (N_v >= 4; N_v <= 4 unless SPC_ANY) -> SPC; otherwise split.
struct TreeBuilder {
    const polar_code *c;
    std::vector<uint32_t> prefix;   // prefix[i] = frozen count in [0, i)
    std::vector<uint32_t> ops, xops;
    std::vector<unsigned long long> desc;
    std::vector<int32_t> sched;
    uint32_t leaves = 0, r0 = 0, r1 = 0, rep = 0, spc = 0;

    uint32_t nfrozen(uint32_t a, uint32_t len) const { return prefix[a + len] - prefix[a]; }

    uint32_t classify(int j, uint32_t start) const {
        const uint32_t nv = 1u << j;
        const uint32_t mode = c->flags & 0xFFu;
        if (mode == POLAR_NO_SPECIAL_NODES && nv > 1) return 0;
        const uint32_t nf = nfrozen(start, nv);
        if (nf == nv) return OP_R0;
        if (nf == 0) return OP_R1;
        if (nv >= 2 && nf == nv - 1 && !c->frozen[start + nv - 1]) return OP_REP;
        if (nv >= 4 && nf == 1 && c->frozen[start] && (mode == POLAR_SPC_ANY || nv <= 4)) return OP_SPC;
        return 0;
    }

    // one entry of the fully unrolled schedule
    void expand(uint32_t kind, int j, uint32_t dest, uint32_t start) {
        xops.push_back(op_make(kind, (uint32_t)j, dest));
        static const int32_t ext[7] = {0, 1, 2, 11, 12, 13, 14};
        sched.push_back(ext[kind]);
        sched.push_back(1 << j);
        sched.push_back((int32_t)start);
        if (kind >= OP_R0) {
            ++leaves;
            r0 += kind == OP_R0; r1 += kind == OP_R1; rep += kind == OP_REP; spc += kind == OP_SPC;
        }
    }

    // candidates a forking leaf generates per source path (log2)
    uint32_t log_cands(uint32_t kind, int j) const {
        if (kind == OP_R1) return j == 0 ? 1u : 2u;
        if (kind == OP_REP) return 1u;
        if (kind == OP_SPC) return c->L == 2 ? 1u : 3u;
        return 0u;
    }

    void walk_sub(int j, uint32_t start, uint32_t dest, std::vector<uint32_t> &types, uint32_t &logm, bool &fork) {
        const uint32_t t = classify(j, start);
        if (t) {
            types.push_back(t);
            expand(t, j, dest, start);
            if (t != OP_R0) { fork = true; logm += log_cands(t, j); }
            return;
        }
        types.push_back(0);
        const uint32_t h = 1u << (j - 1);
        expand(OP_F, j, 0, start);
        walk_sub(j - 1, start, 0, types, logm, fork);
        expand(OP_G, j, 0, start);
        walk_sub(j - 1, start + h, 1, types, logm, fork);
        expand(OP_COMB, j, dest, start);
    }

    uint32_t push_desc(const std::vector<uint32_t> &types) {
        unsigned long long w[2] = {0ull, 0ull};
        for (size_t i = 0; i < types.size(); ++i) w[i / 21] |= (unsigned long long)types[i] << (3 * (i % 21));
        const uint32_t di = (uint32_t)(desc.size() / 2);
        desc.push_back(w[0]);
        desc.push_back(w[1]);
        return di;
    }

    void build(int j, uint32_t start, uint32_t dest) {
        if (j <= kSubLog) {
            std::vector<uint32_t> types;
            uint32_t logm = 0;
            bool fork = false;
            walk_sub(j, start, dest, types, logm, fork);
            const uint32_t di = push_desc(types);
            ops.push_back(op_make(OP_SUB, (uint32_t)j, dest) | (fork ? 1u << 11 : 0u) | (std::min(logm, 6u) << 12) |
                          (di << 15));
            return;
        }
        if (j == kSubLog + 1 && c->n > (uint32_t)j && classify(j, start) == 0) {
            // an inner node of 2^(kSubLog+1) bits below the root: F, both
            // register subtrees, G and Combine as one operation (descriptors
            // of the left and right subtree stored consecutively)
            const uint32_t h = 1u << (j - 1);
            std::vector<uint32_t> tl, tr;
            uint32_t logm = 0;
            bool fork = false;
            expand(OP_F, j, 0, start);
            walk_sub(j - 1, start, 0, tl, logm, fork);
            expand(OP_G, j, 0, start);
            walk_sub(j - 1, start + h, 1, tr, logm, fork);
            expand(OP_COMB, j, dest, start);
            const uint32_t di = push_desc(tl);
            push_desc(tr);
            ops.push_back(op_make(OP_SUB, (uint32_t)j, dest) | (fork ? 1u << 11 : 0u) | (std::min(logm, 6u) << 12) |
                          (di << 15));
            return;
        }
        const uint32_t t = classify(j, start);
        if (t) {
            expand(t, j, dest, start);
            ops.push_back(op_make(t, (uint32_t)j, dest));
            return;
        }
        const uint32_t h = 1u << (j - 1);
        expand(OP_F, j, 0, start);
        ops.push_back(op_with_start(op_make(OP_F, (uint32_t)j, 0), start));
        build(j - 1, start, 0);
        expand(OP_G, j, 0, start);
        ops.push_back(op_with_start(op_make(OP_G, (uint32_t)j, 0), start));
        build(j - 1, start + h, 1);
        expand(OP_COMB, j, dest, start);
        ops.push_back(op_make(OP_COMB, (uint32_t)j, dest));
    }
};

// ---- CRC syndrome of every codeword bit ------------------------------------
// The register left after feeding the K information bits of u = x G_N
// (payload then CRC, MSB first, start 0) is zero iff the CRC matches, and it is
// linear in x. Column t is the register for the unit vector at information
// index t; codeword bit i contributes the columns of every information
// position p of row i of G_N, i.e. every p with (p & ~i) == 0. A systematic
// code reads its information bits from x itself: bit i contributes only its
// own column when i is an information position.
void build_syndrome(polar_code *c) {
    const uint32_t K = c->K, N = c->N, cl = c->crc_len;
    const uint32_t mask = cl >= 32 ? 0xffffffffu : ((1u << cl) - 1u);
    const uint32_t poly = (uint32_t)c->crc_poly & mask;
    std::vector<uint32_t> col(K, 0u);
    uint32_t reg = poly;                              // unit vector at index K-1
    for (int t = (int)K - 1; t >= 0; --t) {
        col[t] = reg;
        const uint32_t top = (reg >> (cl - 1)) & 1u;  // one more zero bit fed after it
        reg = ((reg << 1) & mask) ^ (top ? poly : 0u);
    }
    std::vector<uint32_t> T(N, 0u);
    const bool sys = (c->flags & POLAR_SYSTEMATIC) != 0;
    for (uint32_t i = 0; i < N; ++i) {
        uint32_t s = 0;
        for (uint32_t t = 0; t < K; ++t)
            if (sys ? c->info[t] == i : (c->info[t] & ~i) == 0) s ^= col[t];
        T[i] = s;
    }
    c->syn.assign((size_t)(N / 8) * 256, 0u);
    for (uint32_t b = 0; b < N / 8; ++b)
        for (uint32_t v = 0; v < 256; ++v) {
            uint32_t s = 0;
            for (int e = 0; e < 8; ++e)
                if ((v >> e) & 1u) s ^= T[8 * b + e];
            c->syn[(size_t)b * 256 + v] = s;
        }
}

// ---- memory layout of one frame --------------------------------------------
// Small per-path tables always sit in shared memory. Alpha stages and left
// betas exist only for stages kSubLog..n-1 (lower stages stay in registers);
// together with the right/root beta and the channel row they go to shared
// memory until the budget is reached, the largest ones spilling to the
// group's global scratch first.
bool build_layout(uint32_t n, uint32_t L, uint32_t es, uint32_t budget, Layout &lay, uint32_t virt_mask = 0) {
    std::memset(&lay, 0, sizeof(lay));
    const uint32_t N = 1u << n;
    const uint32_t lo = std::min<uint32_t>((uint32_t)kSubLog, n);
    struct Buf { int kind; uint32_t j; uint32_t bytes; bool spill; };
    std::vector<Buf> bufs;
    lay.virt_mask = virt_mask;
    for (uint32_t j = lo; j < n; ++j)
        if (!((virt_mask >> j) & 1u)) bufs.push_back({0, j, al16(L * (1u << j) * es), false});
    for (uint32_t j = lo; j < n; ++j) bufs.push_back({1, j, al16(L * 4u * (uint32_t)beta_words((int)j)), false});
    bufs.push_back({2, 0, al16(L * 4u * (uint32_t)beta_words((int)n)), false});
    bufs.push_back({3, 0, al16(N * es), false});
    const uint32_t fixed = 4 * al16(L * 16u) + 2 * al16(L * 4u) + al16(L * 8u) + al16(4u * (uint32_t)beta_words((int)n));
    uint64_t total = fixed;
    for (const Buf &bf : bufs) total += bf.bytes;
    while (total > budget) {
        int pick = -1;
        for (size_t i = 0; i < bufs.size(); ++i)
            if (!bufs[i].spill && (pick < 0 || bufs[i].bytes > bufs[(size_t)pick].bytes)) pick = (int)i;
        if (pick < 0) return false;
        bufs[(size_t)pick].spill = true;
        total -= bufs[(size_t)pick].bytes;
    }
    uint32_t off = 0;
    uint64_t goff = 0;
    for (const Buf &bf : bufs) {
        uint32_t *so = nullptr;
        uint64_t *go = nullptr;
        if (bf.kind == 0) { so = &lay.alpha[bf.j]; go = &lay.galpha[bf.j]; if (bf.spill) lay.spill_mask |= 1u << bf.j; }
        else if (bf.kind == 1) { so = &lay.bl[bf.j]; go = &lay.gbl[bf.j]; if (bf.spill) lay.bl_spill |= 1u << bf.j; }
        else if (bf.kind == 2) { so = &lay.br; go = &lay.gbr; if (bf.spill) lay.flags |= LAY_BR_GLOBAL; }
        else { so = &lay.chan; go = &lay.gchan; if (bf.spill) lay.flags |= LAY_CHAN_GLOBAL; }
        if (bf.spill) { *go = goff; goff = al256(goff + bf.bytes); }
        else { *so = off; off += bf.bytes; }
    }
    for (int b = 0; b < 2; ++b) { lay.idx[b] = off; off += al16(L * 16u); }
    for (int b = 0; b < 2; ++b) { lay.bidx[b] = off; off += al16(L * 16u); }
    for (int b = 0; b < 2; ++b) { lay.pen[b] = off; off += al16(L * 4u); }
    lay.surv = off; off += al16(L * 8u);
    lay.ubuf = off; off += al16(4u * (uint32_t)beta_words((int)n));
    lay.bytes = off;
    lay.gbytes = goff;
    return true;
}

constexpr uint32_t kMaxSmemPerCta = 232448;   // 227 KB opt-in per CTA on sm_100-class parts

// Solo / sync flags for a group of `warps` warps: leaves and subtrees run on
// warp 0 alone (one lane per path); a group barrier is needed after an
// operation unless it and the next one are both solo.
std::vector<uint32_t> flag_ops(const std::vector<uint32_t> &ops, uint32_t warps) {
    std::vector<uint32_t> out(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) {
        const bool solo = warps == 1 || op_kind(ops[i]) >= OP_R0;
        const bool next_solo = i + 1 < ops.size() && (warps == 1 || op_kind(ops[i + 1]) >= OP_R0);
        out[i] = ops[i] | (solo ? OP_SOLO : 0u) | ((warps > 1 && !(solo && next_solo)) ? OP_SYNC : 0u);
    }
    return out;
}

// Stages n - d .. n - 1, the ones evaluated from the channel at depth d.
uint32_t virt_mask_of(uint32_t n, uint32_t d) { return d == 0 ? 0u : ((1u << d) - 1u) << (n - d); }

bool make_shape(const polar_code *c, int dtype, uint32_t warps, uint32_t budget, LaunchShape &sh,
                uint32_t cta_threads = 0, int vdepth = -1) {
    if (warps != 1 && warps != 2 && warps != 4) return false;
    if (cta_threads == 0) cta_threads = 128;
    if (cta_threads % (32u * warps) != 0 || cta_threads > (uint32_t)kMaxCtaThreads) return false;
    const uint32_t es = dtype == POLAR_LLR_I8 ? 1u : 4u;
    const uint32_t gpc = cta_threads / (32u * warps);
    if (budget == 0) {
        // Default: 4 frames per SM with 4 warps each, 6 with 2, 8 with 1, and
        // never more than one CTA's share of the shared memory.
        const uint32_t groups_per_sm = warps == 4 ? 4u : (warps == 2 ? 6u : 8u);
        budget = (kMaxSmemPerCta / std::max(groups_per_sm, gpc)) & ~15u;
    }
    budget = std::min(budget, kMaxSmemPerCta / gpc);
    const uint32_t vd = vdepth < 0 ? c->vdepth[dtype] : (uint32_t)vdepth;
    if (vd > c->vmax) return false;
    Layout lay;
    if (!build_layout(c->n, c->L, es, budget, lay, virt_mask_of(c->n, vd))) return false;
    sh.d_ops = nullptr;
    sh.budget = budget;
    sh.pack = packs(c, dtype, warps) ? 1 : 0;
    sh.warps = (int)warps;
    sh.groups_per_cta = (int)gpc;
    sh.threads = (int)cta_threads;
    sh.smem = lay.bytes * gpc;
    sh.lay = lay;
    return sh.smem <= kMaxSmemPerCta;
}

uint32_t default_warps(const polar_code *c) {
    const uint64_t ln = (uint64_t)c->L * c->N;
    if (ln >= 16384) return 4;
    if (ln >= 2048) return 2;
    return 1;
}

void free_device(polar_code *c) {
    for (int d = 0; d < 2; ++d) {
        if (c->shape[d].d_ops) cudaFree(c->shape[d].d_ops);
        c->shape[d].d_ops = nullptr;
        if (c->lat[d].d_ops) cudaFree(c->lat[d].d_ops);
        c->lat[d].d_ops = nullptr;
    }
    if (c->d_syn) cudaFree(c->d_syn);
    if (c->d_info) cudaFree(c->d_info);
    if (c->d_desc) cudaFree(c->d_desc);
    if (c->d_xops) cudaFree(c->d_xops);
    c->d_xops = nullptr;
    if (c->d_sops) cudaFree(c->d_sops);
    c->d_sops = nullptr;
    c->d_syn = nullptr;
    c->d_info = nullptr;
    c->d_desc = nullptr;
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &v) {
    cudaError_t e = cudaMalloc((void **)dst, std::max<size_t>(v.size(), 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    if (!v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

// Install a launch shape for one dtype: flag the schedule and upload it.
int install_shape(polar_code *c, int dtype, const LaunchShape &sh) {
    std::vector<uint32_t> fl = flag_ops(c->ops, (uint32_t)sh.warps);
    uint32_t *d = nullptr;
    if (!c->host_only) {
        cudaError_t e = upload(&d, fl);
        if (e != cudaSuccess) {
            if (d) cudaFree(d);
            return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : POLAR_ECUDA;
        }
    }
    if (c->shape[dtype].d_ops) cudaFree(c->shape[dtype].d_ops);
    c->shape[dtype] = sh;
    c->shape[dtype].d_ops = d;
    c->shape_ops[dtype] = std::move(fl);
    return POLAR_OK;
}

CodeView make_view(const polar_code *code, const LaunchShape &sh) {
    CodeView v;
    std::memset(&v, 0, sizeof(v));
    v.ops = sh.d_ops;
    v.syn = code->d_syn;
    v.info = code->d_info;
    v.desc = code->d_desc;
    v.n_ops = (int)code->ops.size();
    v.N = (int)code->N;
    v.n = (int)code->n;
    v.L = (int)code->L;
    v.K = (int)code->K;
    v.k = (int)code->k;
    v.kb = (int)((code->k + 7) / 8);
    v.crc_len = (int)code->crc_len;
    v.systematic = (code->flags & POLAR_SYSTEMATIC) ? 1 : 0;
    v.pack = sh.pack;
    v.lay = sh.lay;
    return v;
}

// Launch a decode of n_frames with an explicit shape.
int decode_shape(const polar_code *code, int dtype, const LaunchShape &sh, const void *llr, uint32_t n_frames,
                 uint8_t *bits, float *pm, uint8_t *ok, int32_t *slot, cudaStream_t st,
                 const uint32_t *frame_idx = nullptr, const uint32_t *frame_cnt = nullptr) {
    int occ = occupancy_locked(dtype, sh);
    if (occ <= 0) return POLAR_ECUDA;
    uint64_t grid = (uint64_t)occ * (uint64_t)code->sm_count;
    const uint64_t need_ctas = ((uint64_t)n_frames + sh.groups_per_cta - 1) / sh.groups_per_cta;
    if (grid > need_ctas) grid = need_ctas;
    Params p;
    std::memset(&p, 0, sizeof(p));
    p.cv = make_view(code, sh);
    p.llr = llr;
    p.bits = bits;
    p.pm = pm;
    p.ok = ok;
    p.slot = slot;
    p.n_frames = n_frames;
    p.groups_per_cta = sh.groups_per_cta;
    p.frame_idx = frame_idx;
    p.frame_cnt = frame_cnt;
    void *scratch = nullptr;
    if (sh.lay.gbytes > 0) {
        const size_t bytes = (size_t)grid * sh.groups_per_cta * sh.lay.gbytes;
        if (scratch_alloc(&scratch, bytes, st) != cudaSuccess) return POLAR_ENOMEM;
        scratch_poison(scratch, bytes, dtype, st);
        p.scratch = (uint8_t *)scratch;
    }
    cudaError_t e = launch_decode_locked(dtype, sh, p, (int)grid, st);
    if (scratch) cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
}

// ---- wide lists ---------------------------------------------------------------
// The CTA's buffers: alpha stages 0..n-1 (L rows of 2^j elements), left betas
// 0..n-1, the right/root beta and the channel row. The smallest go to shared
// memory until `budget` bytes are used (the small stages are the ones the many
// small nodes of the tree touch), the rest to the CTA's global scratch.
WideView &wide_view(const polar_code *c, int dtype, WideView &v, uint32_t budget) {
    std::memset(&v, 0, sizeof(v));
    const uint64_t es = dtype == POLAR_LLR_I8 ? 1 : 4;
    struct Buf { uint64_t *loc; uint64_t bytes; };
    std::vector<Buf> bufs;
    for (uint32_t j = 0; j < c->n; ++j) bufs.push_back({&v.galpha[j], (uint64_t)c->L * (1u << j) * es});
    for (uint32_t j = 0; j < c->n; ++j) bufs.push_back({&v.gbl[j], (uint64_t)c->L * 4u * (uint64_t)beta_words((int)j)});
    bufs.push_back({&v.gbr, (uint64_t)c->L * 4u * (uint64_t)beta_words((int)c->n)});
    bufs.push_back({&v.gchan, (uint64_t)c->N * es});
    std::stable_sort(bufs.begin(), bufs.end(), [](const Buf &a, const Buf &b) { return a.bytes < b.bytes; });
    uint64_t goff = 0;
    uint32_t soff = 0;
    const uint32_t limit = std::min<uint32_t>(budget, kMaxSmemPerCta - wide_smem_bytes((int)c->L, (int)c->n));
    for (const Buf &b : bufs) {
        const uint32_t need = (uint32_t)((b.bytes + 15u) & ~uint64_t(15));
        if (b.bytes <= limit && soff + need <= limit) {
            *b.loc = kWideInSmem | soff;
            soff += need;
        } else {
            *b.loc = goff;
            goff = al256(goff + b.bytes);
        }
    }
    v.sbytes = soff;
    v.gbytes = goff;
    v.xops = c->d_xops;
    v.syn = c->d_syn;
    v.info = c->d_info;
    v.n_xops = (int)c->xops.size();
    v.N = (int)c->N;
    v.n = (int)c->n;
    v.L = (int)c->L;
    v.K = (int)c->K;
    v.k = (int)c->k;
    v.kb = (int)((c->k + 7) / 8);
    v.crc_len = (int)c->crc_len;
    v.systematic = (c->flags & POLAR_SYSTEMATIC) ? 1 : 0;
    return v;
}

int decode_wide(const polar_code *code, int dtype, const void *llr, uint32_t n_frames, uint8_t *bits, float *pm,
                uint8_t *ok, int32_t *slot, cudaStream_t st, const uint32_t *frame_idx, const uint32_t *frame_cnt,
                uint32_t budget = 0) {
    WideParams p;
    std::memset(&p, 0, sizeof(p));
    wide_view(code, dtype, p.v, budget ? budget : code->wide_budget[dtype]);
    const int occ = occupancy_wide(dtype, (int)code->L, wide_smem_bytes((int)code->L, (int)code->n) + p.v.sbytes);
    if (occ <= 0) return POLAR_ECUDA;
    uint64_t grid = (uint64_t)occ * (uint64_t)code->sm_count;
    if (grid > n_frames) grid = n_frames;
    p.llr = llr;
    p.bits = bits;
    p.pm = pm;
    p.ok = ok;
    p.slot = slot;
    p.n_frames = n_frames;
    p.frame_idx = frame_idx;
    p.frame_cnt = frame_cnt;
    void *scratch = nullptr;
    if (p.v.gbytes > 0) {
        if (scratch_alloc(&scratch, (size_t)(grid * p.v.gbytes), st) != cudaSuccess) return POLAR_ENOMEM;
        scratch_poison(scratch, (size_t)(grid * p.v.gbytes), dtype, st);
        p.scratch = (uint8_t *)scratch;
    }
    cudaError_t e = launch_wide(dtype, p, (int)grid, st);
    if (scratch) cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
}

// ---- L = 1 ----------------------------------------------------------------------
bool use_sc1(const polar_code *c, int dtype) { return c->L == 1 && c->d_sops && !c->explicit_shape[dtype]; }

// The L = 1 kernel: 32 frames per warp, one lane each; warps per CTA as many
// as the shared memory takes (at most kSc1Threads / 32).
struct Sc1Shape : Sc1Layout {
    int warps;
    // float codes with special nodes (Fast-SSC) run the instantiation that drops
    // dead spilled stages from L2: measured 2 to 5 % faster; plain SC decoding
    // (one-bit leaves, many more small operations) lost 15 % to it, mostly to
    // the registers it adds, and keeps the plain one
    bool drop;
};

Sc1Shape sc1_shape(const polar_code *code, int dtype, uint32_t budget) {
    Sc1Shape sh;
    const int es = dtype == POLAR_LLR_I8 ? 1 : 4;
    sc1_layout((int)code->n, es, std::min(budget, kMaxSmemPerCta), &sh);
    sh.warps = sh.warp_bytes == 0 ? kSc1Threads / 32
                                  : std::max(1, std::min<int>(kSc1Threads / 32, (int)(kMaxSmemPerCta / sh.warp_bytes)));
    sh.drop = dtype == POLAR_LLR_F32 && (code->flags & 0xFFu) != POLAR_NO_SPECIAL_NODES;
    return sh;
}

Sc1Params sc1_params(const polar_code *code, const Sc1Shape &sh, const void *llr, uint32_t n_frames, uint8_t *bits,
                     float *pm, uint8_t *ok, int32_t *slot, const uint32_t *frame_idx, const uint32_t *frame_cnt) {
    Sc1Params p;
    std::memset(&p, 0, sizeof(p));
    p.ops = code->d_sops;
    p.n_ops = (int)code->sops.size();
    p.syn = code->d_syn;
    p.info = code->d_info;
    p.n = (int)code->n;
    p.k = (int)code->k;
    p.kb = (int)((code->k + 7) / 8);
    p.crc_len = (int)code->crc_len;
    p.systematic = (code->flags & POLAR_SYSTEMATIC) ? 1 : 0;
    p.split = sh.split;
    p.beta_smem = sh.beta_smem;
    p.warp_bytes = sh.warp_bytes;
    p.beta_off = sh.beta_off;
    p.warp_gbytes = sh.warp_gbytes;
    p.drop = sh.drop ? 1 : 0;
    p.llr = llr;
    p.bits = bits;
    p.pm = pm;
    p.ok = ok;
    p.slot = slot;
    p.n_frames = n_frames;
    p.frame_idx = frame_idx;
    p.frame_cnt = frame_cnt;
    return p;
}

// Grid of the L = 1 kernel: resident CTAs, no more than the frames need.
int sc1_grid(const polar_code *code, int dtype, const Sc1Shape &sh, uint32_t n_frames, uint64_t *grid) {
    const int occ = occupancy_sc1_locked(dtype, sh.warp_bytes, sh.warps, sh.drop);
    if (occ <= 0) return POLAR_ECUDA;
    uint64_t g = (uint64_t)occ * (uint64_t)code->sm_count;
    const uint64_t need = ((uint64_t)n_frames + 32u * sh.warps - 1) / (32u * sh.warps);
    if (g > need) g = need;
    *grid = std::max<uint64_t>(g, 1);
    return POLAR_OK;
}

int decode_sc1(const polar_code *code, int dtype, const void *llr, uint32_t n_frames, uint8_t *bits, float *pm,
               uint8_t *ok, int32_t *slot, cudaStream_t st, const uint32_t *frame_idx, const uint32_t *frame_cnt,
               uint32_t budget = 0) {
    const Sc1Shape sh = sc1_shape(code, dtype, budget ? budget : code->sc1_budget[dtype]);
    Sc1Params p = sc1_params(code, sh, llr, n_frames, bits, pm, ok, slot, frame_idx, frame_cnt);
    uint64_t grid = 0;
    const int rc = sc1_grid(code, dtype, sh, n_frames, &grid);
    if (rc != POLAR_OK) return rc;
    void *scratch = nullptr;
    if (sh.warp_gbytes > 0) {
        const size_t bytes = (size_t)grid * sh.warps * sh.warp_gbytes;
        if (scratch_alloc(&scratch, bytes, st) != cudaSuccess) return POLAR_ENOMEM;
        scratch_poison(scratch, bytes, dtype, st);
        p.scratch = (uint8_t *)scratch;
    }
    const cudaError_t e = launch_sc1_locked(dtype, p, (int)grid, sh.warps, st);
    if (scratch) cudaFreeAsync(scratch, st);
    return e == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
}

// L = 1, small batches: one warp per frame, one warp per CTA (so that the
// frames spread over the SMs); nothing in global scratch.
int decode_sc1w(const polar_code *code, int dtype, const void *llr, uint32_t n_frames, uint8_t *bits, float *pm,
                uint8_t *ok, int32_t *slot, cudaStream_t st) {
    Sc1wParams p;
    std::memset(&p, 0, sizeof(p));
    const bool root_leaf = code->sops.size() == 1;
    p.ops = code->d_sops;
    p.n_ops = (int)code->sops.size();
    p.syn = code->d_syn;
    p.info = code->d_info;
    p.n = (int)code->n;
    p.k = (int)code->k;
    p.kb = (int)((code->k + 7) / 8);
    p.crc_len = (int)code->crc_len;
    p.systematic = (code->flags & POLAR_SYSTEMATIC) ? 1 : 0;
    p.root_leaf = root_leaf ? 1 : 0;
    p.warp_bytes = sc1w_warp_bytes((int)code->n, dtype == POLAR_LLR_I8 ? 1 : 4, root_leaf, &p.beta_off);
    p.llr = llr;
    p.bits = bits;
    p.pm = pm;
    p.ok = ok;
    p.slot = slot;
    p.n_frames = n_frames;
    const int occ = occupancy_sc1w_locked(dtype, (int)code->n, root_leaf, 1);
    if (occ <= 0) return POLAR_ECUDA;
    const uint64_t grid = std::min<uint64_t>((uint64_t)occ * (uint64_t)code->sm_count, n_frames);
    return launch_sc1w_locked(dtype, p, (int)std::max<uint64_t>(grid, 1), 1, st) == cudaSuccess ? POLAR_OK
                                                                                                 : POLAR_ECUDA;
}

// The installed shape of the narrow kernels, the L = 1 kernel or the wide kernel.
int decode_any(const polar_code *code, int dtype, const void *llr, uint32_t n_frames, uint8_t *bits, float *pm,
               uint8_t *ok, int32_t *slot, cudaStream_t st, const uint32_t *frame_idx = nullptr,
               const uint32_t *frame_cnt = nullptr) {
    if (code->wide) return decode_wide(code, dtype, llr, n_frames, bits, pm, ok, slot, st, frame_idx, frame_cnt);
    // a batch no larger than the SM count is latency-bound: give each frame a
    // CTA of its own with everything on chip (unless the shape was fixed).
    // At L = 1 that is one warp over the node elements, where one lane would
    // otherwise walk a whole frame alone.
    const bool small = n_frames <= (uint32_t)code->sm_count && !frame_idx;
    if (use_sc1(code, dtype))
        return small ? decode_sc1w(code, dtype, llr, n_frames, bits, pm, ok, slot, st)
                     : decode_sc1(code, dtype, llr, n_frames, bits, pm, ok, slot, st, frame_idx, frame_cnt);
    const LaunchShape &sh = (small && !code->explicit_shape[dtype] && code->lat[dtype].d_ops) ? code->lat[dtype]
                                                                                                : code->shape[dtype];
    return decode_shape(code, dtype, sh, llr, n_frames, bits, pm, ok, slot, st, frame_idx, frame_cnt);
}

// ---- allocation-free decoding ----------------------------------------------
// Some callers cannot allocate device memory while they decode: real-time
// paths that must not take allocator locks or risk an out-of-memory failure
// once they are running, and hosts that hand the decoder a fixed memory
// budget. For them the spilled alpha stages live in one fixed array that is
// part of the library image: every GPU that loads the library holds these
// kNoAllocScratchBytes until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)64 << 20;   // 64 MiB
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the array on the current device. The name of a
// __device__ array in host code is only a host-side stand-in, so the address
// is looked up once per device (with that device current) and cached.
int noalloc_scratch(int device, uint8_t **out) {
    if (device < 0 || device >= kMaxDevices) return POLAR_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return POLAR_ECUDA;
        g_noalloc_ptr[device] = ptr;
    }
    *out = (uint8_t *)g_noalloc_ptr[device];
    return POLAR_OK;
}

}  // namespace

extern "C" {

int polar_sync(polar_stream_t stream) {
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
}

const char *polar_strerror(int status) {
    switch (status) {
        case POLAR_OK: return "ok";
        case POLAR_EINVAL: return "invalid argument";
        case POLAR_ENOMEM: return "out of memory";
        case POLAR_ECUDA: return "CUDA error";
        case POLAR_EUNSUPPORTED: return "unsupported";
        case POLAR_ETIMEDOUT: return "timed out";
        case POLAR_EBUSY: return "busy";
        default: return "unknown status";
    }
}

int polar_code_create(polar_code_t **out, uint32_t N, uint32_t K, const uint8_t *frozen_mask, uint32_t crc_len,
                      uint64_t crc_poly, uint32_t L, uint32_t flags) {
    if (!out) return POLAR_EINVAL;
    *out = nullptr;
    if (!frozen_mask) return POLAR_EINVAL;
    if (N < 8 || N > 4096 || (N & (N - 1))) return POLAR_EINVAL;
    if (K > N || crc_len > 32 || (crc_len > 0 && crc_len >= K) || (crc_len == 0 && K == 0)) return POLAR_EINVAL;
    if ((flags & ~0x3FFu) != 0 || (flags & 0xFFu) > POLAR_NO_SPECIAL_NODES) return POLAR_EINVAL;
    if (L < 1 || L > (uint32_t)kMaxWideL || (L & (L - 1))) return POLAR_EUNSUPPORTED;
    uint32_t nf = 0;
    for (uint32_t i = 0; i < N; ++i) nf += frozen_mask[i] ? 1u : 0u;
    if (nf != N - K) return POLAR_EINVAL;

    polar_code *c = new (std::nothrow) polar_code();
    if (!c) return POLAR_ENOMEM;
    c->N = N;
    c->n = 0;
    while ((1u << c->n) < N) ++c->n;
    c->K = K;
    c->k = K - crc_len;
    c->L = L;
    c->crc_len = crc_len;
    c->crc_poly = crc_poly;
    c->flags = flags;
    c->frozen.assign(frozen_mask, frozen_mask + N);
    for (uint32_t i = 0; i < N; ++i) c->frozen[i] = frozen_mask[i] ? 1 : 0;
    for (uint32_t i = 0; i < N; ++i)
        if (!c->frozen[i]) c->info.push_back((uint16_t)i);

    TreeBuilder tb;
    tb.c = c;
    tb.prefix.assign(N + 1, 0u);
    for (uint32_t i = 0; i < N; ++i) tb.prefix[i + 1] = tb.prefix[i] + c->frozen[i];
    tb.build((int)c->n, 0, 1);
    c->ops = std::move(tb.ops);
    c->xops = std::move(tb.xops);
    c->desc = std::move(tb.desc);
    c->sched = std::move(tb.sched);
    for (size_t i = 0; i < c->xops.size(); ++i)
        c->sops.push_back(sc1_op(op_kind(c->xops[i]), (uint32_t)op_stage(c->xops[i]), (uint32_t)c->sched[3 * i + 2]));
    // stages every node of which is an inner node run by F / G / Combine can be
    // evaluated from the channel (top stages only, at most three, >= kSubLog + 2)
    for (uint32_t d = 1; d <= 3 && d + (uint32_t)kSubLog + 2 <= c->n; ++d) {
        const uint32_t j = c->n - d;
        bool inner = true;
        for (uint32_t op : c->ops) {
            const uint32_t k = op_kind(op);
            if ((uint32_t)op_stage(op) == j && k != OP_F && k != OP_G && k != OP_COMB) inner = false;
        }
        if (!inner) break;
        c->vmax = d;
    }
    // stored by default: measured, evaluating them costs more than it saves
    for (int d = 0; d < 2; ++d) c->vdepth[d] = 0;
    for (int d = 0; d < 2; ++d) c->pack_pref[d] = L <= kPackDefaultMaxL;
    c->n_leaves = tb.leaves;
    c->n_r0 = tb.r0;
    c->n_r1 = tb.r1;
    c->n_rep = tb.rep;
    c->n_spc = tb.spc;
    if (crc_len > 0) build_syndrome(c);
    c->host_only = (flags & POLAR_HOST_ONLY) != 0;
    if (!c->host_only) {
        if (cudaGetDevice(&c->device) != cudaSuccess ||
            cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
            delete c;
            return POLAR_ECUDA;
        }
        cudaError_t e = upload(&c->d_info, c->info);
        if (e == cudaSuccess) e = upload(&c->d_syn, c->syn);
        if (e == cudaSuccess) e = upload(&c->d_desc, c->desc);
        if (e == cudaSuccess && L > (uint32_t)kMaxL) e = upload(&c->d_xops, c->xops);
        if (e == cudaSuccess && L == 1) e = upload(&c->d_sops, c->sops);
        if (e != cudaSuccess) {
            free_device(c);
            delete c;
            return e == cudaErrorMemoryAllocation ? POLAR_ENOMEM : POLAR_ECUDA;
        }
    }
    if (L > (uint32_t)kMaxL) {
        c->wide = true;
        *out = c;
        return POLAR_OK;
    }
    // the latency shape: four warps and every stage that fits in a CTA's
    // shared memory (one warp with the selection in L-lane segments was
    // measured slower for one frame at every L <= 16)
    for (int d = 0; d < 2; ++d) {
        LaunchShape lat;
        if (!c->host_only && make_shape(c, d, 4, 0xffffffffu, lat, 128, 0) &&
            upload(&lat.d_ops, flag_ops(c->ops, 4)) == cudaSuccess)
            c->lat[d] = lat;
    }
    for (int d = 0; d < 2; ++d) {
        LaunchShape sh;
        int st = make_shape(c, d, default_warps(c), 0, sh) ? install_shape(c, d, sh) : POLAR_EUNSUPPORTED;
        if (st != POLAR_OK) {
            free_device(c);
            delete c;
            return st;
        }
    }
    *out = c;
    return POLAR_OK;
}

int polar_code_destroy(polar_code_t *code) {
    if (!code) return POLAR_OK;
    free_device(code);
    delete code;
    return POLAR_OK;
}

int polar_list_decode(const polar_code_t *code, const void *llr_dev, int llr_dtype, uint32_t n_frames,
                      uint8_t *info_bits_dev, float *path_metric_dev, uint8_t *crc_ok_dev, int32_t *winner_slot_dev,
                      polar_stream_t stream) {
    if (!code || code->host_only) return POLAR_EINVAL;
    if (llr_dtype != POLAR_LLR_F32 && llr_dtype != POLAR_LLR_I8) return POLAR_EINVAL;
    if (n_frames == 0) return POLAR_OK;
    if (!llr_dev || !path_metric_dev || (!info_bits_dev && code->k > 0)) return POLAR_EINVAL;
    NvtxRange range("polar_list_decode");
    return decode_any(code, llr_dtype, llr_dev, n_frames, info_bits_dev, path_metric_dev, crc_ok_dev, winner_slot_dev,
                      reinterpret_cast<cudaStream_t>(stream));
}

int polar_list_decode_host(const polar_code_t *code, const void *llr_host, int llr_dtype, uint32_t n_frames,
                           uint8_t *info_bits_host, float *path_metric_host, uint8_t *crc_ok_host,
                           int32_t *winner_slot_host, polar_stream_t stream) {
    if (!code || code->host_only) return POLAR_EINVAL;
    if (llr_dtype != POLAR_LLR_F32 && llr_dtype != POLAR_LLR_I8) return POLAR_EINVAL;
    if (n_frames == 0) return POLAR_OK;
    if (!llr_host || !path_metric_host || (!info_bits_host && code->k > 0)) return POLAR_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return POLAR_ECUDA;
    if (dev != code->device) return POLAR_EINVAL;
    NvtxRange range("polar_list_decode_host");
    const uint64_t row = (uint64_t)code->N * (llr_dtype == POLAR_LLR_I8 ? 1u : 4u);
    const uint64_t kb = (code->k + 7) / 8;
    // chunks of frames in a two-buffer ring: the copy in of chunk c + 1 and the
    // copy out of chunk c - 1 overlap the decode of chunk c. The first chunks
    // are smaller (doubling up to `chunk`) so that the copy in that nothing
    // overlaps is short.
    const uint32_t chunk = std::min<uint32_t>(n_frames, std::max<uint32_t>(4096u, std::min<uint32_t>(131072u, n_frames / 8)));
    const uint32_t first = std::max<uint32_t>(std::min<uint32_t>(chunk, 2048u), chunk / 16u);
    uint32_t n_chunks = 0;
    for (uint64_t f = 0, sz = first; f < n_frames; f += sz, sz = std::min<uint64_t>(2 * sz, chunk)) ++n_chunks;
    const uint64_t out_row = kb + 4 + 1 + 4;
    const uint64_t buf_bytes = (uint64_t)chunk * (row + out_row) + 64;
    cudaStream_t dec = reinterpret_cast<cudaStream_t>(stream);
    cudaStream_t cin = nullptr, cout = nullptr;
    cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_dec[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
    uint8_t *buf[2] = {nullptr, nullptr};
    int rc = POLAR_OK;
    bool ok = cudaStreamCreateWithFlags(&cin, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&cout, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; ok && b < 2; ++b)
        ok = cudaEventCreateWithFlags(&ev_in[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&ev_dec[b], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&ev_out[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) rc = POLAR_ECUDA;
    for (int b = 0; rc == POLAR_OK && b < 2 && b < (int)n_chunks; ++b)
        if (scratch_alloc((void **)&buf[b], buf_bytes, nullptr, false) != cudaSuccess) rc = POLAR_ENOMEM;
    // the caller's stream may have pending work on the host buffers' producers
    if (rc == POLAR_OK && cudaEventRecord(ev_dec[0], dec) != cudaSuccess) rc = POLAR_ECUDA;
    if (rc == POLAR_OK && cudaStreamWaitEvent(cin, ev_dec[0], 0) != cudaSuccess) rc = POLAR_ECUDA;
    uint64_t f0 = 0, sz = first;
    for (uint32_t c = 0; rc == POLAR_OK && c < n_chunks; ++c, f0 += sz, sz = std::min<uint64_t>(2 * sz, chunk)) {
        const int b = (int)(c & 1u);
        const uint32_t nf = (uint32_t)std::min<uint64_t>(sz, n_frames - f0);
        uint8_t *d_llr = buf[b];
        uint8_t *d_bits = d_llr + (uint64_t)chunk * row;
        float *d_pm = reinterpret_cast<float *>(((uintptr_t)(d_bits + (uint64_t)chunk * kb) + 15) & ~(uintptr_t)15);
        int32_t *d_slot = reinterpret_cast<int32_t *>(d_pm + chunk);
        uint8_t *d_ok = reinterpret_cast<uint8_t *>(d_slot + chunk);
        // buffer b is free once the copy out of chunk c - 2 finished
        if (c >= 2 && cudaStreamWaitEvent(cin, ev_out[b], 0) != cudaSuccess) { rc = POLAR_ECUDA; break; }
        if (cudaMemcpyAsync(d_llr, static_cast<const uint8_t *>(llr_host) + f0 * row, (size_t)nf * row,
                            cudaMemcpyHostToDevice, cin) != cudaSuccess ||
            cudaEventRecord(ev_in[b], cin) != cudaSuccess || cudaStreamWaitEvent(dec, ev_in[b], 0) != cudaSuccess) {
            rc = POLAR_ECUDA;
            break;
        }
        rc = decode_any(code, llr_dtype, d_llr, nf, d_bits, d_pm, d_ok, d_slot, dec);
        if (rc != POLAR_OK) break;
        if (cudaEventRecord(ev_dec[b], dec) != cudaSuccess || cudaStreamWaitEvent(cout, ev_dec[b], 0) != cudaSuccess) {
            rc = POLAR_ECUDA;
            break;
        }
        bool cp = true;
        if (code->k > 0)
            cp = cudaMemcpyAsync(info_bits_host + f0 * kb, d_bits, (size_t)nf * kb, cudaMemcpyDeviceToHost, cout) ==
                 cudaSuccess;
        cp = cp && cudaMemcpyAsync(path_metric_host + f0, d_pm, (size_t)nf * 4, cudaMemcpyDeviceToHost, cout) ==
                       cudaSuccess;
        if (crc_ok_host)
            cp = cp && cudaMemcpyAsync(crc_ok_host + f0, d_ok, nf, cudaMemcpyDeviceToHost, cout) == cudaSuccess;
        if (winner_slot_host)
            cp = cp && cudaMemcpyAsync(winner_slot_host + f0, d_slot, (size_t)nf * 4, cudaMemcpyDeviceToHost, cout) ==
                           cudaSuccess;
        if (!cp || cudaEventRecord(ev_out[b], cout) != cudaSuccess) { rc = POLAR_ECUDA; break; }
    }
    // drain everything that was enqueued, also after an error
    if (cin && cudaStreamSynchronize(cin) != cudaSuccess) rc = POLAR_ECUDA;
    if (cudaStreamSynchronize(dec) != cudaSuccess) rc = POLAR_ECUDA;
    if (cout && cudaStreamSynchronize(cout) != cudaSuccess) rc = POLAR_ECUDA;
    for (int b = 0; b < 2; ++b) {
        if (buf[b]) cudaFree(buf[b]);
        if (ev_in[b]) cudaEventDestroy(ev_in[b]);
        if (ev_dec[b]) cudaEventDestroy(ev_dec[b]);
        if (ev_out[b]) cudaEventDestroy(ev_out[b]);
    }
    if (cin) cudaStreamDestroy(cin);
    if (cout) cudaStreamDestroy(cout);
    return rc;
}

int polar_adaptive_decode(const polar_code_t *fast, const polar_code_t *list, const void *llr_dev, int llr_dtype,
                          uint32_t n_frames, uint8_t *info_bits_dev, float *path_metric_dev, uint8_t *crc_ok_dev,
                          int32_t *winner_slot_dev, uint32_t *n_relisted_dev, polar_stream_t stream) {
    if (!fast || !list || fast->host_only || list->host_only) return POLAR_EINVAL;
    if (fast->N != list->N || fast->K != list->K || fast->crc_len != list->crc_len ||
        fast->crc_poly != list->crc_poly || fast->frozen != list->frozen || fast->device != list->device)
        return POLAR_EINVAL;
    if (fast->crc_len == 0) return POLAR_EINVAL;   // the switch is driven by the CRC
    if (llr_dtype != POLAR_LLR_F32 && llr_dtype != POLAR_LLR_I8) return POLAR_EINVAL;
    if (n_frames == 0) return POLAR_OK;
    if (!llr_dev || !path_metric_dev || !crc_ok_dev || (!info_bits_dev && fast->k > 0)) return POLAR_EINVAL;
    NvtxRange range("polar_adaptive_decode");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = decode_any(fast, llr_dtype, llr_dev, n_frames, info_bits_dev, path_metric_dev, crc_ok_dev,
                        winner_slot_dev, st);
    if (rc != POLAR_OK) return rc;
    void *tmp = nullptr;
    if (scratch_alloc(&tmp, sizeof(uint32_t) * ((size_t)n_frames + 1), st) != cudaSuccess) return POLAR_ENOMEM;
    uint32_t *cnt = (uint32_t *)tmp;
    uint32_t *idx = cnt + 1;
    if (launch_crc_failures(crc_ok_dev, n_frames, idx, cnt, st) != cudaSuccess) {
        cudaFreeAsync(tmp, st);
        return POLAR_ECUDA;
    }
    if (n_relisted_dev && cudaMemcpyAsync(n_relisted_dev, cnt, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) !=
                              cudaSuccess) {
        cudaFreeAsync(tmp, st);
        return POLAR_ECUDA;
    }
    rc = decode_any(list, llr_dtype, llr_dev, n_frames, info_bits_dev, path_metric_dev, crc_ok_dev, winner_slot_dev,
                    st, idx, cnt);
    cudaFreeAsync(tmp, st);
    return rc;
}

int polar_code_autotune(polar_code_t *code, int llr_dtype, const void *llr_dev, uint32_t n_frames,
                        polar_stream_t stream, uint32_t *warps_out, uint32_t *budget_out, uint32_t *cta_out) {
    if (!code || code->host_only || !llr_dev || n_frames == 0) return POLAR_EINVAL;
    if (llr_dtype != POLAR_LLR_F32 && llr_dtype != POLAR_LLR_I8) return POLAR_EINVAL;
    if (code->wide) {
        // a CTA of L threads per frame: time how much shared memory its
        // smallest buffers get (more on chip against fewer CTAs per SM)
        static const uint32_t wide_budgets[] = {1u, 8000u, 16000u, 24000u, 36000u, 48000u, 64000u, 96000u,
                                                140000u, kMaxSmemPerCta};
        cudaStream_t stw = reinterpret_cast<cudaStream_t>(stream);
        const size_t kbw = (code->k + 7) / 8;
        uint8_t *bw = nullptr;
        float *pmw = nullptr;
        if (cudaMalloc(&bw, std::max<size_t>(kbw, 1) * n_frames) != cudaSuccess) return POLAR_ENOMEM;
        if (cudaMalloc(&pmw, sizeof(float) * n_frames) != cudaSuccess) {
            cudaFree(bw);
            return POLAR_ENOMEM;
        }
        cudaEvent_t aw, zw;
        cudaEventCreate(&aw);
        cudaEventCreate(&zw);
        float bestw = 1e30f;
        uint32_t bestb = code->wide_budget[llr_dtype];
        uint32_t last_sbytes = 0xffffffffu;
        int statusw = POLAR_OK;
        for (uint32_t b : wide_budgets) {
            WideView wv;
            wide_view(code, llr_dtype, wv, b);
            if (wv.sbytes == last_sbytes) continue;               // the same placement as the last budget
            last_sbytes = wv.sbytes;
            int rc = decode_wide(code, llr_dtype, llr_dev, n_frames, bw, pmw, nullptr, nullptr, stw, nullptr, nullptr, b);
            float ms = 0.f;
            if (rc == POLAR_OK) {
                cudaEventRecord(aw, stw);
                rc = decode_wide(code, llr_dtype, llr_dev, n_frames, bw, pmw, nullptr, nullptr, stw, nullptr, nullptr, b);
                cudaEventRecord(zw, stw);
                if (cudaEventSynchronize(zw) != cudaSuccess) { statusw = POLAR_ECUDA; break; }
                cudaEventElapsedTime(&ms, aw, zw);
            }
            if (rc == POLAR_ENOMEM) { statusw = rc; break; }
            if (rc == POLAR_OK && ms < bestw) { bestw = ms; bestb = b; }
        }
        cudaEventDestroy(aw);
        cudaEventDestroy(zw);
        cudaFree(bw);
        cudaFree(pmw);
        if (statusw != POLAR_OK) return statusw;
        code->wide_budget[llr_dtype] = bestb;
        if (warps_out) *warps_out = code->L / 32;
        if (budget_out) *budget_out = bestb;
        if (cta_out) *cta_out = code->L;
        return POLAR_OK;
    }
    if (code->L == 1 && code->d_sops) {
        // the L = 1 kernel: time the shared-memory budgets per warp (how many
        // alpha stages stay on chip against how many warps fit) and keep the fastest
        static const uint32_t sc1_budgets[] = {0u, 9000u, 17000u, 25000u, 33000u, 46000u, 57000u, 76000u,
                                               112000u, kMaxSmemPerCta};
        // A sample that does not fill every SM at the default layout would
        // favour layouts with fewer resident warps; keep the default then.
        {
            const Sc1Shape d0 = sc1_shape(code, llr_dtype, 0);
            const int occ0 = occupancy_sc1_locked(llr_dtype, d0.warp_bytes, d0.warps, d0.drop);
            if (occ0 <= 0) return POLAR_ECUDA;
            if ((uint64_t)n_frames < (uint64_t)occ0 * code->sm_count * 32u * (uint64_t)d0.warps) {
                code->sc1_budget[llr_dtype] = 0;
                code->explicit_shape[llr_dtype] = false;
                if (warps_out) *warps_out = 1;
                if (budget_out) *budget_out = 0;
                if (cta_out) *cta_out = 32u * (uint32_t)d0.warps;
                return POLAR_OK;
            }
        }
        cudaStream_t st1 = reinterpret_cast<cudaStream_t>(stream);
        const size_t kb1 = (code->k + 7) / 8;
        uint8_t *b1 = nullptr;
        float *pm1 = nullptr;
        if (cudaMalloc(&b1, std::max<size_t>(kb1, 1) * n_frames) != cudaSuccess) return POLAR_ENOMEM;
        if (cudaMalloc(&pm1, sizeof(float) * n_frames) != cudaSuccess) {
            cudaFree(b1);
            return POLAR_ENOMEM;
        }
        cudaEvent_t a1, z1;
        cudaEventCreate(&a1);
        cudaEventCreate(&z1);
        float best1 = 1e30f;
        uint32_t bestb = 0;
        int seen_split = -2;
        int status1 = POLAR_OK;
        for (uint32_t b : sc1_budgets) {
            const Sc1Shape shp = sc1_shape(code, llr_dtype, b);
            const int key = shp.beta_smem ? shp.split : -1;
            if (key == seen_split) continue;                // the same layout as the last budget
            seen_split = key;
            int rc = decode_sc1(code, llr_dtype, llr_dev, n_frames, b1, pm1, nullptr, nullptr, st1, nullptr, nullptr, b);
            float ms = 0.f;
            if (rc == POLAR_OK) {
                cudaEventRecord(a1, st1);
                rc = decode_sc1(code, llr_dtype, llr_dev, n_frames, b1, pm1, nullptr, nullptr, st1, nullptr, nullptr, b);
                cudaEventRecord(z1, st1);
                if (cudaEventSynchronize(z1) != cudaSuccess) { status1 = POLAR_ECUDA; break; }
                cudaEventElapsedTime(&ms, a1, z1);
            }
            if (rc == POLAR_ENOMEM) { status1 = rc; break; }
            if (rc == POLAR_OK && ms < best1) { best1 = ms; bestb = b; }
        }
        cudaEventDestroy(a1);
        cudaEventDestroy(z1);
        cudaFree(b1);
        cudaFree(pm1);
        if (status1 != POLAR_OK) return status1;
        code->sc1_budget[llr_dtype] = bestb;
        code->explicit_shape[llr_dtype] = false;
        const Sc1Shape fin = sc1_shape(code, llr_dtype, bestb);
        if (warps_out) *warps_out = 1;
        if (budget_out) *budget_out = bestb;
        if (cta_out) *cta_out = 32u * (uint32_t)fin.warps;
        return POLAR_OK;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t kb = (code->k + 7) / 8;
    uint8_t *bits = nullptr;
    float *pm = nullptr;
    if (cudaMalloc(&bits, std::max<size_t>(kb, 1) * n_frames) != cudaSuccess) return POLAR_ENOMEM;
    if (cudaMalloc(&pm, sizeof(float) * n_frames) != cudaSuccess) {
        cudaFree(bits);
        return POLAR_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    static const uint32_t budgets[] = {0xffffffffu, 110000u, 75000u, 56000u, 44000u, 36000u, 28000u, 20000u,
                                       14000u, 10000u, 7000u};
    float best_ms = 1e30f;
    LaunchShape best;
    uint32_t best_w = 0, best_b = 0, best_t = 0;
    std::vector<std::array<uint32_t, 5>> seen;   // (warps, CTA threads, spill masks, depth) already timed
    int status = POLAR_OK;
    uint32_t best_vd = 0;
    // every shape with all stages stored, then the best one with 1 .. vmax
    // top stages evaluated from the channel
    for (uint32_t vd = 0; vd <= code->vmax && status == POLAR_OK; ++vd) {
    for (uint32_t w : {4u, 2u, 1u}) {
      for (uint32_t t : {128u, 256u, 512u}) {
        for (uint32_t b : budgets) {
            if (vd > 0 && (w != best_w || t != best_t || b != best_b)) continue;
            LaunchShape sh;
            if (!make_shape(code, llr_dtype, w, b, sh, t, (int)vd)) continue;
            bool dup = false;
            for (auto &pr : seen)
                dup |= pr[0] == w && pr[1] == t && pr[2] == sh.lay.spill_mask && pr[3] == sh.lay.flags &&
                       pr[4] == vd;
            if (dup) continue;
            seen.push_back({w, t, sh.lay.spill_mask, sh.lay.flags, vd});
            std::vector<uint32_t> fl = flag_ops(code->ops, w);
            if (upload(&sh.d_ops, fl) != cudaSuccess) { status = POLAR_ECUDA; break; }
            float ms = 0.f;
            int rc = decode_shape(code, llr_dtype, sh, llr_dev, n_frames, bits, pm, nullptr, nullptr, st);
            if (rc == POLAR_OK) {
                cudaEventRecord(e0, st);
                rc = decode_shape(code, llr_dtype, sh, llr_dev, n_frames, bits, pm, nullptr, nullptr, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = POLAR_ECUDA;
                cudaEventElapsedTime(&ms, e0, e1);
            }
            cudaFree(sh.d_ops);
            sh.d_ops = nullptr;
            if (rc != POLAR_OK) continue;
            if (ms < best_ms) { best_ms = ms; best = sh; best_w = w; best_b = b; best_t = t; best_vd = vd; }
        }
        if (status != POLAR_OK) break;
      }
      if (status != POLAR_OK) break;
    }
    }
    // several frames' register subtrees to a warp (L <= 16, one warp per frame,
    // 32 / L frame groups to a CTA) on the best shape
    if (status == POLAR_OK && best_w == 1 && code->L <= 16) {
        LaunchShape sh = best;
        sh.pack = best.pack ^ 1;
        std::vector<uint32_t> fl = flag_ops(code->ops, 1);
        if (upload(&sh.d_ops, fl) == cudaSuccess) {
            float ms = 0.f;
            int rc = decode_shape(code, llr_dtype, sh, llr_dev, n_frames, bits, pm, nullptr, nullptr, st);
            if (rc == POLAR_OK) {
                cudaEventRecord(e0, st);
                rc = decode_shape(code, llr_dtype, sh, llr_dev, n_frames, bits, pm, nullptr, nullptr, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = POLAR_ECUDA;
                cudaEventElapsedTime(&ms, e0, e1);
            }
            cudaFree(sh.d_ops);
            sh.d_ops = nullptr;
            if (rc == POLAR_OK && ms < best_ms) { best_ms = ms; best = sh; }
        }
    }
    if (status == POLAR_OK && best_w == 1 && code->L <= 16) code->pack_pref[llr_dtype] = best.pack != 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(bits);
    cudaFree(pm);
    if (status != POLAR_OK) return status;
    if (best_w == 0) return POLAR_ECUDA;
    if (warps_out) *warps_out = best_w;
    if (budget_out) *budget_out = best_b == 0xffffffffu ? 0u : best_b;
    if (cta_out) *cta_out = best_t;
    code->explicit_shape[llr_dtype] = false;
    code->vdepth[llr_dtype] = best_vd;
    return install_shape(code, llr_dtype, best);
}

int polar_list_decode_noalloc(const polar_code_t *code, const void *llr_dev, int llr_dtype, uint32_t n_frames,
                              uint8_t *info_bits_dev, float *path_metric_dev, uint8_t *crc_ok_dev,
                              int32_t *winner_slot_dev, polar_stream_t stream) {
    if (!code || code->host_only) return POLAR_EINVAL;
    if (code->wide) return POLAR_EUNSUPPORTED;
    if (llr_dtype != POLAR_LLR_F32 && llr_dtype != POLAR_LLR_I8) return POLAR_EINVAL;
    if (n_frames == 0) return POLAR_OK;
    if (!llr_dev || !path_metric_dev || (!info_bits_dev && code->k > 0)) return POLAR_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return POLAR_ECUDA;
    if (dev != code->device) return POLAR_EINVAL;
    if (use_sc1(code, llr_dtype)) {
        // the L = 1 kernel: its spilled stages go to the fixed array too, the
        // persistent grid cut to what the array holds
        const Sc1Shape s1 = sc1_shape(code, llr_dtype, code->sc1_budget[llr_dtype]);
        Sc1Params p1 = sc1_params(code, s1, llr_dev, n_frames, info_bits_dev, path_metric_dev, crc_ok_dev,
                                  winner_slot_dev, nullptr, nullptr);
        uint64_t g1 = 0;
        const int rc1 = sc1_grid(code, llr_dtype, s1, n_frames, &g1);
        if (rc1 != POLAR_OK) return rc1;
        const uint64_t per_cta1 = (uint64_t)s1.warps * s1.warp_gbytes;
        if (per_cta1 > 0) {
            if (per_cta1 > kNoAllocScratchBytes) return POLAR_EUNSUPPORTED;
            g1 = std::min<uint64_t>(g1, kNoAllocScratchBytes / per_cta1);
            uint8_t *scr = nullptr;
            const int st1 = noalloc_scratch(dev, &scr);
            if (st1 != POLAR_OK) return st1;
            scratch_poison(scr, (size_t)(g1 * per_cta1), llr_dtype, reinterpret_cast<cudaStream_t>(stream));
            p1.scratch = scr;
        }
        const cudaError_t e1 = launch_sc1_locked(llr_dtype, p1, (int)g1, s1.warps,
                                                 reinterpret_cast<cudaStream_t>(stream));
        return e1 == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
    }
    const LaunchShape &sh = code->shape[llr_dtype];
    const int occ = occupancy_locked(llr_dtype, sh);
    if (occ <= 0) return POLAR_ECUDA;
    uint64_t grid = (uint64_t)occ * (uint64_t)code->sm_count;
    const uint64_t need_ctas = ((uint64_t)n_frames + sh.groups_per_cta - 1) / sh.groups_per_cta;
    if (grid > need_ctas) grid = need_ctas;
    uint8_t *scratch = nullptr;
    const uint64_t per_cta = (uint64_t)sh.groups_per_cta * sh.lay.gbytes;
    if (per_cta > 0) {
        // The kernel is persistent, so fewer CTAs still decode every frame;
        // a shape whose single CTA needs more than the array is refused.
        if (per_cta > kNoAllocScratchBytes) return POLAR_EUNSUPPORTED;
        const uint64_t fit = kNoAllocScratchBytes / per_cta;
        if (grid > fit) grid = fit;
        const int st = noalloc_scratch(dev, &scratch);
        if (st != POLAR_OK) return st;
        scratch_poison(scratch, (size_t)(grid * per_cta), llr_dtype, reinterpret_cast<cudaStream_t>(stream));
    }
    Params p;
    std::memset(&p, 0, sizeof(p));
    p.cv = make_view(code, sh);
    p.llr = llr_dev;
    p.bits = info_bits_dev;
    p.pm = path_metric_dev;
    p.ok = crc_ok_dev;
    p.slot = winner_slot_dev;
    p.n_frames = n_frames;
    p.groups_per_cta = sh.groups_per_cta;
    p.scratch = scratch;
    const cudaError_t e = launch_decode_locked(llr_dtype, sh, p, (int)grid, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
}

size_t polar_noalloc_scratch_bytes(void) { return kNoAllocScratchBytes; }

int polar_debug_inject(int what, int64_t value) {
    if (what == POLAR_INJECT_ALLOC_FAIL) {
        g_fail_alloc_after.store(value < 0 ? -1 : value);
        return POLAR_OK;
    }
    if (what == POLAR_INJECT_POISON) {
        g_poison.store(value != 0 ? 1 : 0);
        return POLAR_OK;
    }
    return POLAR_EINVAL;
}

// ---- batched form ------------------------------------------------------------
struct polar_batch {
    int dtype = 0;
    int device = -1;
    int sm_count = 0;
    uint32_t n_frames = 0;
    std::vector<const polar_code *> codes;
    std::vector<uint32_t> frame_code;
    std::vector<uint64_t> llr_off, bits_off;
    uint64_t llr_bytes = 0, bits_bytes = 0;
    // current launch shape
    int warps = 4;
    uint32_t budget = 0;
    int threads = 128;
    int groups_per_cta = 1;
    uint32_t group_bytes = 0, view_bytes = 0, cta_smem = 0;
    uint64_t gbytes = 0;
    int grid = 0;
    int pack = 1;                      // classes follow their codes' packing choice (0: none packs)
    bool seg = false;                  // some class packs: launch the kernels that hold that code
    // device state
    std::vector<uint32_t *> d_ops;     // per class, flagged for `warps`
    CodeView *d_classes = nullptr;
    BatchItem *d_items = nullptr;
    uint32_t *d_counter = nullptr;
    uint8_t *d_scratch = nullptr;
    uint64_t scratch_bytes = 0;
    cudaGraphExec_t graph = nullptr;
};

namespace {

void batch_free_shape(polar_batch *b) {
    for (uint32_t *p : b->d_ops) if (p) cudaFree(p);
    b->d_ops.clear();
    if (b->d_classes) cudaFree(b->d_classes);
    if (b->d_scratch) cudaFree(b->d_scratch);
    b->d_classes = nullptr;
    b->d_scratch = nullptr;
    b->scratch_bytes = 0;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

// Lay out every class for `warps` warps per frame and a shared-memory budget
// per frame, upload the class table and size the global scratch.
int batch_shape(polar_batch *b, int warps, uint32_t budget, uint32_t cta_threads = 0) {
    if (warps != 1 && warps != 2 && warps != 4) return POLAR_EINVAL;
    if (cta_threads == 0) cta_threads = 128;
    if (cta_threads % (32u * (uint32_t)warps) != 0 || cta_threads > (uint32_t)kMaxCtaThreads) return POLAR_EINVAL;
    const int gpc = (int)cta_threads / (32 * warps);
    const uint32_t view_bytes = al16((uint32_t)sizeof(CodeView) + 16u);
    if (budget == 0) budget = (kMaxSmemPerCta / (warps == 4 ? 4u : (warps == 2 ? 6u : 8u))) & ~15u;
    budget = std::min<uint32_t>(budget, kMaxSmemPerCta / gpc - view_bytes);
    const uint32_t es = b->dtype == POLAR_LLR_I8 ? 1u : 4u;
    std::vector<CodeView> views(b->codes.size());
    uint32_t gb = 0;
    uint64_t gs = 0;
    bool seg = false;
    for (size_t c = 0; c < b->codes.size(); ++c) {
        Layout lay;
        if (!build_layout(b->codes[c]->n, b->codes[c]->L, es, budget, lay)) return POLAR_EINVAL;
        LaunchShape sh;
        std::memset(&sh, 0, sizeof(sh));
        sh.lay = lay;
        sh.pack = b->pack && packs(b->codes[c], b->dtype, (uint32_t)warps) ? 1 : 0;
        seg |= sh.pack != 0;
        views[c] = make_view(b->codes[c], sh);
        gb = std::max(gb, lay.bytes);
        gs = std::max<uint64_t>(gs, lay.gbytes);
    }
    const uint32_t group_bytes = view_bytes + gb;
    const uint32_t cta_smem = group_bytes * (uint32_t)gpc;
    if (cta_smem > kMaxSmemPerCta) return POLAR_EINVAL;
    const int occ = occupancy_batch_locked(b->dtype, warps, seg, cta_smem, (int)cta_threads);
    if (occ <= 0) return POLAR_ECUDA;
    batch_free_shape(b);
    for (size_t c = 0; c < b->codes.size(); ++c) {
        uint32_t *d = nullptr;
        if (upload(&d, flag_ops(b->codes[c]->ops, (uint32_t)warps)) != cudaSuccess) return POLAR_ECUDA;
        b->d_ops.push_back(d);
        views[c].ops = d;
    }
    if (upload(&b->d_classes, views) != cudaSuccess) return POLAR_ECUDA;
    uint64_t grid = (uint64_t)occ * (uint64_t)b->sm_count;
    const uint64_t need = ((uint64_t)b->n_frames + gpc - 1) / gpc;
    if (grid > need) grid = need;
    if (grid == 0) grid = 1;
    b->scratch_bytes = grid * (uint64_t)gpc * gs;
    if (b->scratch_bytes > 0) {
        if (cudaMalloc(&b->d_scratch, b->scratch_bytes) != cudaSuccess) return POLAR_ENOMEM;
    }
    b->warps = warps;
    b->seg = seg;
    b->budget = budget;
    b->threads = (int)cta_threads;
    b->groups_per_cta = gpc;
    b->group_bytes = group_bytes;
    b->view_bytes = view_bytes;
    b->cta_smem = cta_smem;
    b->gbytes = gs;
    b->grid = (int)grid;
    return POLAR_OK;
}

int batch_launch(polar_batch *b, const void *llr, uint8_t *bits, float *pm, uint8_t *ok, int32_t *slot,
                 cudaStream_t st) {
    if (cudaMemsetAsync(b->d_counter, 0, sizeof(uint32_t), st) != cudaSuccess) return POLAR_ECUDA;
    scratch_poison(b->d_scratch, b->scratch_bytes, b->dtype, st);
    BatchParams p;
    std::memset(&p, 0, sizeof(p));
    p.classes = b->d_classes;
    p.items = b->d_items;
    p.n_items = b->n_frames;
    p.counter = b->d_counter;
    p.llr = (const uint8_t *)llr;
    p.bits = bits;
    p.pm = pm;
    p.ok = ok;
    p.slot = slot;
    p.scratch = b->d_scratch;
    p.gbytes = b->gbytes;
    p.group_bytes = b->group_bytes;
    p.view_bytes = b->view_bytes;
    p.groups_per_cta = b->groups_per_cta;
    const cudaError_t e = launch_batch_locked(b->dtype, b->warps, b->seg, p, b->grid, b->cta_smem, b->threads, st);
    return e == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
}

}  // namespace

int polar_batch_plan(polar_batch_t **out, polar_code_t *const *codes, uint32_t n_codes, const uint32_t *frame_code,
                     uint32_t n_frames, int llr_dtype, uint32_t flags) {
    if (!out) return POLAR_EINVAL;
    *out = nullptr;
    if (!codes || n_codes == 0 || (!frame_code && n_frames > 0) || flags != 0) return POLAR_EINVAL;
    if (llr_dtype != POLAR_LLR_F32 && llr_dtype != POLAR_LLR_I8) return POLAR_EINVAL;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return POLAR_ECUDA;
    for (uint32_t c = 0; c < n_codes; ++c)
        if (!codes[c] || codes[c]->host_only || codes[c]->device != dev) return POLAR_EINVAL;
    for (uint32_t c = 0; c < n_codes; ++c)
        if (codes[c]->wide) return POLAR_EUNSUPPORTED;
    for (uint32_t f = 0; f < n_frames; ++f)
        if (frame_code[f] >= n_codes) return POLAR_EINVAL;
    polar_batch *b = new (std::nothrow) polar_batch();
    if (!b) return POLAR_ENOMEM;
    b->dtype = llr_dtype;
    b->device = dev;
    b->sm_count = codes[0]->sm_count;
    b->n_frames = n_frames;
    b->codes.assign(codes, codes + n_codes);
    b->frame_code.assign(frame_code, frame_code + n_frames);
    const uint64_t es = llr_dtype == POLAR_LLR_I8 ? 1 : 4;
    b->llr_off.resize(n_frames);
    b->bits_off.resize(n_frames);
    for (uint32_t f = 0; f < n_frames; ++f) {
        const polar_code *c = codes[frame_code[f]];
        b->llr_off[f] = b->llr_bytes;
        b->bits_off[f] = b->bits_bytes;
        b->llr_bytes += (uint64_t)c->N * es;
        b->bits_bytes += (c->k + 7) / 8;
    }
    // work items: classes by decreasing cost, frames in order within a class
    std::vector<uint64_t> cost(n_codes, 0);
    for (uint32_t c = 0; c < n_codes; ++c) polar_code_op_count(codes[c], &cost[c]);
    std::vector<uint32_t> order(n_codes);
    for (uint32_t c = 0; c < n_codes; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t x) { return cost[a] > cost[x]; });
    std::vector<std::vector<uint32_t>> per(n_codes);
    for (uint32_t f = 0; f < n_frames; ++f) per[frame_code[f]].push_back(f);
    std::vector<BatchItem> items;
    items.reserve(n_frames);
    for (uint32_t c : order)
        for (uint32_t f : per[c]) items.push_back(BatchItem{c, f, b->llr_off[f], b->bits_off[f]});
    int st = POLAR_OK;
    if (upload(&b->d_items, items) != cudaSuccess || cudaMalloc(&b->d_counter, sizeof(uint32_t)) != cudaSuccess)
        st = POLAR_ENOMEM;
    if (st == POLAR_OK) st = batch_shape(b, 4, 0);
    if (st != POLAR_OK) {
        polar_batch_destroy(b);
        return st;
    }
    *out = b;
    return POLAR_OK;
}

int polar_batch_destroy(polar_batch_t *b) {
    if (!b) return POLAR_OK;
    batch_free_shape(b);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_counter) cudaFree(b->d_counter);
    delete b;
    return POLAR_OK;
}

int polar_batch_layout(const polar_batch_t *b, uint64_t *llr_bytes, uint64_t *bits_bytes, uint64_t *llr_offsets,
                       uint64_t *bits_offsets) {
    if (!b) return POLAR_EINVAL;
    if (llr_bytes) *llr_bytes = b->llr_bytes;
    if (bits_bytes) *bits_bytes = b->bits_bytes;
    if (llr_offsets) std::memcpy(llr_offsets, b->llr_off.data(), b->llr_off.size() * sizeof(uint64_t));
    if (bits_offsets) std::memcpy(bits_offsets, b->bits_off.data(), b->bits_off.size() * sizeof(uint64_t));
    return POLAR_OK;
}

int polar_batch_run(polar_batch_t *b, const void *llr_dev, uint8_t *bits_dev, float *pm_dev, uint8_t *ok_dev,
                    int32_t *slot_dev, polar_stream_t stream) {
    if (!b || (b->n_frames > 0 && (!llr_dev || !pm_dev || !bits_dev))) return POLAR_EINVAL;
    if (b->n_frames == 0) return POLAR_OK;
    NvtxRange range("polar_batch_run");
    return batch_launch(b, llr_dev, bits_dev, pm_dev, ok_dev, slot_dev, reinterpret_cast<cudaStream_t>(stream));
}

int polar_batch_set_launch(polar_batch_t *b, uint32_t warps_per_frame, uint32_t smem_budget, uint32_t cta_threads) {
    if (!b) return POLAR_EINVAL;
    return batch_shape(b, (int)warps_per_frame, smem_budget, cta_threads);
}

int polar_batch_autotune(polar_batch_t *b, const void *llr_dev, uint8_t *bits_dev, float *pm_dev,
                         polar_stream_t stream, uint32_t *warps_out, uint32_t *budget_out, uint32_t *cta_out) {
    if (!b || !llr_dev || !bits_dev || !pm_dev) return POLAR_EINVAL;
    if (b->n_frames == 0) return POLAR_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a coarser grid than the plain form's: every timing runs the whole plan
    static const uint32_t budgets[] = {0u, 28000u, 14000u, 7000u};
    float best = 1e30f;
    int bw = 0;
    uint32_t bb = 0, bt = 0;
    for (int w : {2, 1}) {
      for (uint32_t t : {128u, 256u, 512u}) {
        for (uint32_t bud : budgets) {
            if (batch_shape(b, w, bud, t) != POLAR_OK) continue;
            if (batch_launch(b, llr_dev, bits_dev, pm_dev, nullptr, nullptr, st) != POLAR_OK) continue;
            cudaEventRecord(e0, st);
            const int rc = batch_launch(b, llr_dev, bits_dev, pm_dev, nullptr, nullptr, st);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || rc != POLAR_OK) continue;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; bw = w; bb = bud; bt = t; }
        }
      }
    }
    // the other packing choice on the best shape
    if (bw == 1) {
        const int keep = b->pack;
        b->pack = keep ^ 1;
        float ms = 0.f;
        int rc = batch_shape(b, bw, bb, bt);
        if (rc == POLAR_OK) rc = batch_launch(b, llr_dev, bits_dev, pm_dev, nullptr, nullptr, st);
        if (rc == POLAR_OK) {
            cudaEventRecord(e0, st);
            rc = batch_launch(b, llr_dev, bits_dev, pm_dev, nullptr, nullptr, st);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = POLAR_ECUDA;
            cudaEventElapsedTime(&ms, e0, e1);
        }
        if (rc != POLAR_OK || ms >= best) b->pack = keep;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bw == 0) return POLAR_ECUDA;
    if (warps_out) *warps_out = (uint32_t)bw;
    if (budget_out) *budget_out = bb;
    if (cta_out) *cta_out = bt;
    return batch_shape(b, bw, bb, bt);
}

int polar_batch_capture(polar_batch_t *b, const void *llr_dev, uint8_t *bits_dev, float *pm_dev, uint8_t *ok_dev,
                        int32_t *slot_dev, polar_stream_t stream) {
    if (!b || b->n_frames == 0 || !llr_dev || !bits_dev || !pm_dev) return POLAR_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (!st) return POLAR_EINVAL;       // the legacy default stream cannot be captured
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return POLAR_ECUDA;
    const int rc = batch_launch(b, llr_dev, bits_dev, pm_dev, ok_dev, slot_dev, st);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &g);
    if (rc != POLAR_OK || ec != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return POLAR_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    return ei == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
}

int polar_batch_replay(polar_batch_t *b, polar_stream_t stream) {
    if (!b || !b->graph) return POLAR_EINVAL;
    return cudaGraphLaunch(b->graph, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? POLAR_OK : POLAR_ECUDA;
}

int polar_batch_get_info(const polar_batch_t *b, polar_batch_info_t *info) {
    if (!b || !info) return POLAR_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->n_frames = b->n_frames;
    info->n_codes = (uint32_t)b->codes.size();
    info->warps_per_frame = (uint32_t)b->warps;
    info->frames_per_cta = (uint32_t)b->groups_per_cta;
    info->smem_per_frame = b->group_bytes;
    info->grid = (uint32_t)b->grid;
    info->scratch_bytes = b->scratch_bytes;
    info->llr_bytes = b->llr_bytes;
    info->bits_bytes = b->bits_bytes;
    return POLAR_OK;
}

int polar_code_get_info(const polar_code_t *c, polar_code_info_t *info) {
    if (!c || !info) return POLAR_EINVAL;
    std::memset(info, 0, sizeof(*info));
    info->N = c->N;
    info->K = c->K;
    info->k = c->k;
    info->L = c->L;
    info->crc_len = c->crc_len;
    info->n_ops = (uint32_t)c->xops.size();
    info->n_leaves = c->n_leaves;
    info->n_rate0 = c->n_r0;
    info->n_rate1 = c->n_r1;
    info->n_rep = c->n_rep;
    info->n_spc = c->n_spc;
    for (int d = 0; d < 2; ++d) {
        if (c->wide) {
            info->warps_per_frame[d] = c->L / 32;
            info->frames_per_cta[d] = 1;
            WideView wv;
            wide_view(c, d, wv, c->wide_budget[d]);
            info->smem_per_frame[d] = wide_smem_bytes((int)c->L, (int)c->n) + wv.sbytes;
            info->scratch_per_frame[d] = wv.gbytes;
            uint32_t sm = 0;
            for (uint32_t j = 0; j < c->n; ++j)
                if (!(wv.galpha[j] & kWideInSmem)) sm |= 1u << j;
            info->spill_mask[d] = sm;
            continue;
        }
        if (c->L == 1 && !c->explicit_shape[d]) {
            // one lane per frame: a warp decodes 32 frames
            const Sc1Shape s1 = sc1_shape(c, d, c->sc1_budget[d]);
            info->warps_per_frame[d] = 1;
            info->frames_per_cta[d] = 32u * (uint32_t)s1.warps;
            info->smem_per_frame[d] = s1.warp_bytes / 32u;
            info->scratch_per_frame[d] = s1.warp_gbytes / 32u;
            info->spill_mask[d] = ((1u << c->n) - 1u) & ~((1u << s1.split) - 1u);
            continue;
        }
        info->warps_per_frame[d] = (uint32_t)c->shape[d].warps;
        info->frames_per_cta[d] = (uint32_t)c->shape[d].groups_per_cta;
        info->smem_per_frame[d] = c->shape[d].lay.bytes;
        info->scratch_per_frame[d] = c->shape[d].lay.gbytes;
        info->spill_mask[d] = c->shape[d].lay.spill_mask;
        info->recomputed_stages[d] = c->shape[d].lay.virt_mask;
        info->packed[d] = c->shape[d].pack ? 1u : 0u;
    }
    info->max_recompute_depth = c->vmax;
    return POLAR_OK;
}

int polar_code_schedule(const polar_code_t *c, int32_t *ops_out, uint32_t cap, uint32_t *n_ops) {
    if (!c || !n_ops) return POLAR_EINVAL;
    const uint32_t cnt = (uint32_t)(c->sched.size() / 3);
    *n_ops = cnt;
    if (!ops_out || cap < cnt) return POLAR_EINVAL;
    std::memcpy(ops_out, c->sched.data(), c->sched.size() * sizeof(int32_t));
    return POLAR_OK;
}

int polar_code_op_count(const polar_code_t *c, uint64_t *ops_per_frame) {
    if (!c || !ops_per_frame) return POLAR_EINVAL;
    uint64_t tot = 0, la = 1;
    uint64_t lg = 0;
    while ((1u << lg) < c->L) ++lg;
    if (lg == 0) lg = 1;
    for (uint32_t op : c->xops) {
        const uint32_t kind = op_kind(op);
        const uint64_t nv = 1ull << op_stage(op);
        switch (kind) {
            case OP_F:
            case OP_G: tot += 2 * (nv / 2) * la; break;
            case OP_COMB: tot += std::max<uint64_t>(1, nv / 64) * la; break;
            case OP_R0: tot += 2 * nv * la; break;
            default: {
                uint64_t C;
                if (kind == OP_R1) { tot += 3 * nv * la; C = nv == 1 ? 2 : 4; }
                else if (kind == OP_REP) { tot += 4 * nv * la; C = 2; }
                else { tot += 5 * nv * la; C = c->L == 2 ? 2 : 8; }
                if (C * la > c->L) tot += C * la * lg;
                la = std::min<uint64_t>(c->L, C * la);
            }
        }
    }
    tot += (uint64_t)c->L * c->N * c->n / 32 + (uint64_t)c->L * c->K;
    *ops_per_frame = tot;
    return POLAR_OK;
}

int polar_code_set_smem_budget(polar_code_t *c, int llr_dtype, uint32_t bytes) {
    if (!c || (llr_dtype != POLAR_LLR_F32 && llr_dtype != POLAR_LLR_I8)) return POLAR_EINVAL;
    if (c->wide) {
        c->wide_budget[llr_dtype] = bytes ? bytes : kWideDefaultBudget;
        return POLAR_OK;
    }
    if (c->L != 1) return POLAR_EUNSUPPORTED;
    c->sc1_budget[llr_dtype] = bytes;
    c->explicit_shape[llr_dtype] = false;
    return POLAR_OK;
}

int polar_code_set_packing(polar_code_t *c, int llr_dtype, int on) {
    if (!c || (llr_dtype != POLAR_LLR_F32 && llr_dtype != POLAR_LLR_I8)) return POLAR_EINVAL;
    if (c->wide) return POLAR_EUNSUPPORTED;
    LaunchShape sh = c->shape[llr_dtype];
    if (on && (sh.warps != 1 || c->L > 16)) return POLAR_EINVAL;
    sh.pack = on ? 1 : 0;
    sh.d_ops = nullptr;
    const bool fixed = c->explicit_shape[llr_dtype];
    const int st = install_shape(c, llr_dtype, sh);
    c->explicit_shape[llr_dtype] = fixed;
    if (st == POLAR_OK) c->pack_pref[llr_dtype] = on != 0;
    return st;
}

int polar_code_set_recompute(polar_code_t *c, int llr_dtype, uint32_t depth) {
    if (!c || (llr_dtype != POLAR_LLR_F32 && llr_dtype != POLAR_LLR_I8)) return POLAR_EINVAL;
    if (c->wide) return POLAR_EUNSUPPORTED;
    if (depth > c->vmax) return POLAR_EINVAL;
    LaunchShape sh;
    const LaunchShape &cur = c->shape[llr_dtype];
    if (!make_shape(c, llr_dtype, (uint32_t)cur.warps, cur.budget, sh, (uint32_t)cur.threads, (int)depth))
        return POLAR_EINVAL;
    const int st = install_shape(c, llr_dtype, sh);
    if (st == POLAR_OK) c->vdepth[llr_dtype] = depth;
    return st;
}

int polar_code_set_launch(polar_code_t *c, int llr_dtype, uint32_t warps_per_frame, uint32_t smem_budget,
                          uint32_t cta_threads) {
    if (!c || (llr_dtype != POLAR_LLR_F32 && llr_dtype != POLAR_LLR_I8)) return POLAR_EINVAL;
    if (c->wide) return POLAR_EUNSUPPORTED;
    LaunchShape sh;
    if (!make_shape(c, llr_dtype, warps_per_frame, smem_budget, sh, cta_threads)) return POLAR_EINVAL;
    const int st = install_shape(c, llr_dtype, sh);
    if (st == POLAR_OK) c->explicit_shape[llr_dtype] = true;
    return st;
}

}  // extern "C"

// ---- serving form (continuous batching) ---------------------------------------
namespace {

double now_us() {
    return (double)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count() * 1e-3;
}

// First-fit allocator over [0, size) with coalescing.
struct RangeAlloc {
    std::map<uint64_t, uint64_t> free_;
    void init(uint64_t size) {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(uint64_t sz, uint64_t &off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= sz) {
                off = it->first;
                const uint64_t rem = it->second - sz, o2 = it->first + sz;
                free_.erase(it);
                if (rem) free_[o2] = rem;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t sz) {
        if (!sz) return;
        auto it = free_.emplace(off, sz).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct SrvReq {
    uint64_t ticket = 0;
    const polar_code *code = nullptr;
    int dtype = 0;
    uint32_t n = 0;
    std::vector<uint8_t> llr;                 // host copy taken at submit
    uint64_t arena_off = 0, arena_sz = 0, llr_sz = 0, bits_sz = 0;
    uint64_t fslot = 0;                       // first frame slot
    std::vector<uint8_t> bits, ok;
    std::vector<float> pm;
    bool done = false;
    double t_submit = 0.0, t_done = 0.0;
};

constexpr int kSrvStreams = 3;
constexpr uint32_t kSrvMaxCodes = 512;

}  // namespace

struct polar_server {
    int device = -1, sm_count = 0;
    uint64_t arena_bytes = 0;
    uint32_t max_frames = 0, max_pending = 0;
    int warps = 4;
    uint32_t smem_budget = 0;
    uint8_t *d_arena = nullptr, *h_arena = nullptr;
    float *d_pm = nullptr, *h_pm = nullptr;
    uint8_t *d_ok = nullptr, *h_ok = nullptr;
    RangeAlloc arena, frames;
    // registered codes: one class table per dtype
    std::vector<const polar_code *> codes;
    std::unordered_map<const polar_code *, uint32_t> code_idx;
    std::vector<uint32_t *> class_ops;
    std::vector<uint8_t> class_pack[2];       // per class and LLR type: its view packs
    CodeView *d_classes[2] = {nullptr, nullptr};
    uint32_t frame_bytes[2] = {0, 0};         // largest per-frame shared layout
    uint64_t gbytes[2] = {0, 0};              // largest per-frame global scratch
    // streams, each with one batch in flight at most
    cudaStream_t streams[kSrvStreams] = {};
    cudaEvent_t done_ev[kSrvStreams] = {};
    bool busy[kSrvStreams] = {};
    std::vector<SrvReq *> batch[kSrvStreams];
    uint32_t *d_counters = nullptr;
    uint8_t *d_scratch[kSrvStreams] = {};
    uint64_t scratch_sz[kSrvStreams] = {};
    BatchItem *d_items[kSrvStreams] = {}, *h_items[kSrvStreams] = {};
    uint64_t items_cap[kSrvStreams] = {};
    // queues
    std::mutex mu;
    std::condition_variable cv;
    std::deque<SrvReq *> pending, admitted;
    std::unordered_map<uint64_t, SrvReq *> reqs;
    uint64_t next_ticket = 1;
    bool stop = false, paused = false;
    int error = POLAR_OK;
    std::thread worker;
    // statistics since the last reset
    std::vector<double> lat_us;
    std::vector<uint32_t> lat_frames;         // frames of the request of each lat_us entry
    uint64_t frames_done = 0, bits_done = 0, batches = 0, max_inflight = 0;
    double t_first = 0.0, t_last = 0.0;
};

namespace {

// Register a code: its class views (both dtypes) for the server's launch shape.
int srv_register(polar_server *s, const polar_code *c, uint32_t &idx) {
    auto it = s->code_idx.find(c);
    if (it != s->code_idx.end()) { idx = it->second; return POLAR_OK; }
    if (s->codes.size() >= kSrvMaxCodes || c->wide) return POLAR_EUNSUPPORTED;
    uint32_t *ops = nullptr;
    if (upload(&ops, flag_ops(c->ops, (uint32_t)s->warps)) != cudaSuccess) return POLAR_ECUDA;
    idx = (uint32_t)s->codes.size();
    for (int d = 0; d < 2; ++d) {
        Layout lay;
        if (!build_layout(c->n, c->L, d == POLAR_LLR_I8 ? 1u : 4u, s->smem_budget, lay)) {
            cudaFree(ops);
            return POLAR_EUNSUPPORTED;
        }
        LaunchShape sh;
        std::memset(&sh, 0, sizeof(sh));
        sh.lay = lay;
        sh.d_ops = ops;
        sh.pack = packs(c, d, (uint32_t)s->warps) ? 1 : 0;
        CodeView v = make_view(c, sh);
        if (cudaMemcpy(s->d_classes[d] + idx, &v, sizeof(v), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(ops);
            return POLAR_ECUDA;
        }
        s->frame_bytes[d] = std::max(s->frame_bytes[d], lay.bytes);
        if (lay.gbytes > s->gbytes[d]) s->gbytes[d] = lay.gbytes;
    }
    s->codes.push_back(c);
    s->class_ops.push_back(ops);
    for (int d = 0; d < 2; ++d) s->class_pack[d].push_back(packs(c, d, (uint32_t)s->warps) ? 1 : 0);
    s->code_idx[c] = idx;
    return POLAR_OK;
}

uint32_t srv_view_bytes() { return al16((uint32_t)sizeof(CodeView) + 16u); }

// Shared memory per CTA and grid for a dtype's batches.
// Server launches: 256-thread CTAs (lockstep units of up to 8 frames of one code).
constexpr int kSrvCtaThreads = 256;

void srv_shape(const polar_server *s, int d, uint32_t &group_bytes, uint32_t &cta_smem, int &gpc) {
    gpc = kSrvCtaThreads / (32 * s->warps);
    group_bytes = srv_view_bytes() + s->frame_bytes[d];
    cta_smem = group_bytes * (uint32_t)gpc;
}

// Admit a pending request if its memory fits: copy its LLRs to the pinned
// mirror of its arena region (the copy to the device goes with its batch).
bool srv_admit(polar_server *s, SrvReq *r) {
    uint32_t idx;
    if (srv_register(s, r->code, idx) != POLAR_OK) return false;
    const uint64_t es = r->dtype == POLAR_LLR_I8 ? 1 : 4;
    r->llr_sz = (uint64_t)r->n * r->code->N * es;
    r->bits_sz = (uint64_t)r->n * ((r->code->k + 7) / 8);
    r->arena_sz = ((r->llr_sz + 255) & ~uint64_t(255)) + ((r->bits_sz + 255) & ~uint64_t(255));
    uint64_t off = 0, fs = 0;
    if (!s->arena.alloc(r->arena_sz, off)) return false;
    if (!s->frames.alloc(r->n, fs)) {
        s->arena.release(off, r->arena_sz);
        return false;
    }
    r->arena_off = off;
    r->fslot = fs;
    std::memcpy(s->h_arena + off, r->llr.data(), r->llr_sz);
    return true;
}

int srv_grow_scratch(polar_server *s, int stream, uint64_t need) {
    if (need <= s->scratch_sz[stream]) return POLAR_OK;
    if (s->d_scratch[stream]) {
        cudaStreamSynchronize(s->streams[stream]);
        cudaFree(s->d_scratch[stream]);
        s->d_scratch[stream] = nullptr;
        s->scratch_sz[stream] = 0;
    }
    if (cudaMalloc(&s->d_scratch[stream], need) != cudaSuccess) return POLAR_ENOMEM;
    s->scratch_sz[stream] = need;
    return POLAR_OK;
}

// Launch every admitted request of one dtype as one batch on stream i.
int srv_launch(polar_server *s, int i) {
    const int d = s->admitted.front()->dtype;
    std::vector<SrvReq *> take;
    std::deque<SrvReq *> rest;
    for (SrvReq *r : s->admitted) {
        if (r->dtype == d) take.push_back(r);
        else rest.push_back(r);
    }
    s->admitted.swap(rest);
    uint64_t n_items = 0;
    for (SrvReq *r : take) n_items += r->n;
    if (n_items > s->items_cap[i]) {
        if (s->d_items[i]) cudaFree(s->d_items[i]);
        if (s->h_items[i]) cudaFreeHost(s->h_items[i]);
        s->d_items[i] = nullptr;
        s->h_items[i] = nullptr;
        s->items_cap[i] = 0;
        const uint64_t cap = std::max<uint64_t>(n_items, 4096);
        if (cudaMalloc(&s->d_items[i], cap * sizeof(BatchItem)) != cudaSuccess ||
            cudaMallocHost(&s->h_items[i], cap * sizeof(BatchItem)) != cudaSuccess)
            return POLAR_ENOMEM;
        s->items_cap[i] = cap;
    }
    // items: larger codes first, each code's frames adjacent (lockstep units)
    std::vector<SrvReq *> ord = take;
    std::stable_sort(ord.begin(), ord.end(), [s](SrvReq *a, SrvReq *b) {
        const uint64_t ca = (uint64_t)a->code->N * a->code->L, cb = (uint64_t)b->code->N * b->code->L;
        if (ca != cb) return ca > cb;
        return s->code_idx.at(a->code) < s->code_idx.at(b->code);
    });
    const uint64_t es = d == POLAR_LLR_I8 ? 1 : 4;
    uint64_t t = 0;
    for (SrvReq *r : ord) {
        const uint32_t cls = s->code_idx[r->code];
        const uint64_t kb = (r->code->k + 7) / 8;
        const uint64_t bits_base = r->arena_off + ((r->llr_sz + 255) & ~uint64_t(255));
        for (uint32_t f = 0; f < r->n; ++f)
            s->h_items[i][t++] = BatchItem{cls, (uint32_t)(r->fslot + f), r->arena_off + (uint64_t)f * r->code->N * es,
                                           bits_base + f * kb};
    }
    cudaStream_t st = s->streams[i];
    uint32_t group_bytes, cta_smem;
    int gpc;
    srv_shape(s, d, group_bytes, cta_smem, gpc);
    bool seg = false;              // some request of the batch packs
    for (SrvReq *r : take) seg |= s->class_pack[d][s->code_idx[r->code]] != 0;
    const int occ = occupancy_batch_locked(d, s->warps, seg, cta_smem, kSrvCtaThreads);
    if (occ <= 0) return POLAR_ECUDA;
    uint64_t grid = (uint64_t)occ * s->sm_count;
    const uint64_t need = (n_items + gpc - 1) / gpc;
    if (grid > need) grid = need;
    int rc = srv_grow_scratch(s, i, (uint64_t)occ * s->sm_count * gpc * s->gbytes[d]);
    if (rc != POLAR_OK) return rc;
    bool okc = cudaMemcpyAsync(s->d_items[i], s->h_items[i], n_items * sizeof(BatchItem), cudaMemcpyHostToDevice,
                               st) == cudaSuccess;
    for (SrvReq *r : take)
        okc &= cudaMemcpyAsync(s->d_arena + r->arena_off, s->h_arena + r->arena_off, r->llr_sz, cudaMemcpyHostToDevice,
                               st) == cudaSuccess;
    okc &= cudaMemsetAsync(s->d_counters + i, 0, sizeof(uint32_t), st) == cudaSuccess;
    BatchParams p;
    std::memset(&p, 0, sizeof(p));
    p.classes = s->d_classes[d];
    p.items = s->d_items[i];
    p.n_items = (uint32_t)n_items;
    p.counter = s->d_counters + i;
    p.llr = s->d_arena;
    p.bits = s->d_arena;
    p.pm = s->d_pm;
    p.ok = s->d_ok;
    p.slot = nullptr;
    p.scratch = s->d_scratch[i];
    p.gbytes = s->gbytes[d];
    p.group_bytes = group_bytes;
    p.view_bytes = srv_view_bytes();
    p.groups_per_cta = gpc;
    okc &= launch_batch_locked(d, s->warps, seg, p, (int)grid, cta_smem, kSrvCtaThreads, st) == cudaSuccess;
    for (SrvReq *r : take) {
        const uint64_t bits_base = r->arena_off + ((r->llr_sz + 255) & ~uint64_t(255));
        okc &= cudaMemcpyAsync(s->h_arena + bits_base, s->d_arena + bits_base, r->bits_sz, cudaMemcpyDeviceToHost,
                               st) == cudaSuccess;
        okc &= cudaMemcpyAsync(s->h_pm + r->fslot, s->d_pm + r->fslot, r->n * sizeof(float), cudaMemcpyDeviceToHost,
                               st) == cudaSuccess;
        okc &= cudaMemcpyAsync(s->h_ok + r->fslot, s->d_ok + r->fslot, r->n, cudaMemcpyDeviceToHost, st) ==
               cudaSuccess;
    }
    okc &= cudaEventRecord(s->done_ev[i], st) == cudaSuccess;
    s->busy[i] = true;
    s->batch[i] = take;
    ++s->batches;
    uint64_t inflight = 0;
    for (int q = 0; q < kSrvStreams; ++q) inflight += s->busy[q] ? 1u : 0u;
    s->max_inflight = std::max(s->max_inflight, inflight);
    return okc ? POLAR_OK : POLAR_ECUDA;
}

void srv_finish(polar_server *s, int i) {
    const double t = now_us();
    for (SrvReq *r : s->batch[i]) {
        const uint64_t bits_base = r->arena_off + ((r->llr_sz + 255) & ~uint64_t(255));
        r->bits.assign(s->h_arena + bits_base, s->h_arena + bits_base + r->bits_sz);
        r->pm.assign(s->h_pm + r->fslot, s->h_pm + r->fslot + r->n);
        r->ok.assign(s->h_ok + r->fslot, s->h_ok + r->fslot + r->n);
        s->arena.release(r->arena_off, r->arena_sz);
        s->frames.release(r->fslot, r->n);
        r->llr.clear();
        r->llr.shrink_to_fit();
        r->done = true;
        r->t_done = t;
        s->lat_us.push_back(t - r->t_submit);
        s->lat_frames.push_back(r->n);
        s->frames_done += r->n;
        s->bits_done += (uint64_t)r->n * r->code->k;
        if (s->t_first == 0.0 || r->t_submit < s->t_first) s->t_first = r->t_submit;
        s->t_last = t;
    }
    s->batch[i].clear();
    s->busy[i] = false;
}

void srv_engine(polar_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        bool progress = false;
        for (int i = 0; i < kSrvStreams; ++i) {
            if (!s->busy[i]) continue;
            const cudaError_t q = cudaEventQuery(s->done_ev[i]);
            if (q == cudaSuccess) {
                srv_finish(s, i);
                progress = true;
            } else if (q != cudaErrorNotReady) {
                s->error = POLAR_ECUDA;
                s->stop = true;
            }
        }
        if (progress) s->cv.notify_all();
        if (!s->paused) {
            while (!s->pending.empty() && srv_admit(s, s->pending.front())) {
                s->admitted.push_back(s->pending.front());
                s->pending.pop_front();
                progress = true;
            }
            for (int i = 0; i < kSrvStreams && !s->admitted.empty(); ++i) {
                if (s->busy[i]) continue;
                const int rc = srv_launch(s, i);
                if (rc != POLAR_OK) {
                    s->error = rc;
                    s->stop = true;
                    break;
                }
                progress = true;
            }
        }
        if (!progress) s->cv.wait_for(lk, std::chrono::microseconds(40));
    }
    s->cv.notify_all();
}

void srv_free(polar_server *s) {
    for (int i = 0; i < kSrvStreams; ++i) {
        if (s->streams[i]) cudaStreamSynchronize(s->streams[i]);
        if (s->d_scratch[i]) cudaFree(s->d_scratch[i]);
        if (s->d_items[i]) cudaFree(s->d_items[i]);
        if (s->h_items[i]) cudaFreeHost(s->h_items[i]);
        if (s->done_ev[i]) cudaEventDestroy(s->done_ev[i]);
        if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
    }
    for (uint32_t *p : s->class_ops) cudaFree(p);
    for (int d = 0; d < 2; ++d) if (s->d_classes[d]) cudaFree(s->d_classes[d]);
    if (s->d_counters) cudaFree(s->d_counters);
    if (s->d_arena) cudaFree(s->d_arena);
    if (s->h_arena) cudaFreeHost(s->h_arena);
    if (s->d_pm) cudaFree(s->d_pm);
    if (s->h_pm) cudaFreeHost(s->h_pm);
    if (s->d_ok) cudaFree(s->d_ok);
    if (s->h_ok) cudaFreeHost(s->h_ok);
    for (auto &kv : s->reqs) delete kv.second;
    s->reqs.clear();
}

}  // namespace

extern "C" {

int polar_server_create(polar_server_t **out, size_t device_mem_budget, uint32_t max_frames_in_flight,
                        uint32_t warps_per_frame, uint32_t smem_budget, uint32_t flags) {
    if (!out) return POLAR_EINVAL;
    *out = nullptr;
    if (device_mem_budget < 4096 || max_frames_in_flight == 0 || (flags & ~POLAR_SERVER_PAUSED)) return POLAR_EINVAL;
    if (warps_per_frame == 0) warps_per_frame = 1;
    if (warps_per_frame != 1 && warps_per_frame != 2 && warps_per_frame != 4) return POLAR_EINVAL;
    polar_server *s = new (std::nothrow) polar_server();
    if (!s) return POLAR_ENOMEM;
    s->warps = (int)warps_per_frame;
    const uint32_t gpc = (uint32_t)kSrvCtaThreads / (32u * warps_per_frame);
    const uint32_t cap = kMaxSmemPerCta / gpc - al16((uint32_t)sizeof(CodeView) + 16u);
    // default: one warp per frame with a small shared-memory share (larger
    // stages in scratch), the shape that gives the mixed request stream of the
    // benchmark its lowest p50 / p99 latency (four lockstep groups per CTA)
    s->smem_budget = smem_budget ? std::min(smem_budget, cap)
                                 : std::min(cap, warps_per_frame == 1 ? 7000u
                                                                     : (kMaxSmemPerCta / (warps_per_frame == 4 ? 4u : 6u)) & ~15u);
    s->arena_bytes = device_mem_budget;
    s->max_frames = max_frames_in_flight;
    s->max_pending = 1u << 16;
    s->paused = (flags & POLAR_SERVER_PAUSED) != 0;
    int st = POLAR_OK;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess)
        st = POLAR_ECUDA;
    if (st == POLAR_OK &&
        (cudaMalloc(&s->d_arena, device_mem_budget) != cudaSuccess ||
         cudaMallocHost(&s->h_arena, device_mem_budget) != cudaSuccess ||
         cudaMalloc(&s->d_pm, sizeof(float) * max_frames_in_flight) != cudaSuccess ||
         cudaMallocHost(&s->h_pm, sizeof(float) * max_frames_in_flight) != cudaSuccess ||
         cudaMalloc(&s->d_ok, max_frames_in_flight) != cudaSuccess ||
         cudaMallocHost(&s->h_ok, max_frames_in_flight) != cudaSuccess ||
         cudaMalloc(&s->d_counters, sizeof(uint32_t) * kSrvStreams) != cudaSuccess ||
         cudaMalloc(&s->d_classes[0], sizeof(CodeView) * kSrvMaxCodes) != cudaSuccess ||
         cudaMalloc(&s->d_classes[1], sizeof(CodeView) * kSrvMaxCodes) != cudaSuccess))
        st = POLAR_ENOMEM;
    for (int i = 0; st == POLAR_OK && i < kSrvStreams; ++i) {
        if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->done_ev[i], cudaEventDisableTiming) != cudaSuccess)
            st = POLAR_ECUDA;
    }
    if (st != POLAR_OK) {
        srv_free(s);
        delete s;
        return st;
    }
    s->arena.init(device_mem_budget);
    s->frames.init(max_frames_in_flight);
    s->worker = std::thread(srv_engine, s);
    *out = s;
    return POLAR_OK;
}

int polar_server_destroy(polar_server_t *s) {
    if (!s) return POLAR_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    srv_free(s);
    delete s;
    return POLAR_OK;
}

int polar_server_submit(polar_server_t *s, const polar_code_t *code, const void *llr_host, int llr_dtype,
                        uint32_t n_frames, uint64_t *ticket) {
    if (!s || !code || code->host_only || !llr_host || !ticket || n_frames == 0) return POLAR_EINVAL;
    if (llr_dtype != POLAR_LLR_F32 && llr_dtype != POLAR_LLR_I8) return POLAR_EINVAL;
    if (code->device != s->device) return POLAR_EINVAL;
    const uint64_t es = llr_dtype == POLAR_LLR_I8 ? 1 : 4;
    const uint64_t llr_sz = (uint64_t)n_frames * code->N * es;
    const uint64_t need = ((llr_sz + 255) & ~uint64_t(255)) + (((uint64_t)n_frames * ((code->k + 7) / 8) + 255) & ~uint64_t(255));
    if (need > s->arena_bytes || n_frames > s->max_frames) return POLAR_EINVAL;   // can never fit
    SrvReq *r = new (std::nothrow) SrvReq();
    if (!r) return POLAR_ENOMEM;
    r->code = code;
    r->dtype = llr_dtype;
    r->n = n_frames;
    r->llr.assign((const uint8_t *)llr_host, (const uint8_t *)llr_host + llr_sz);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->error != POLAR_OK) {
            delete r;
            return s->error;
        }
        if (s->pending.size() >= s->max_pending) {
            delete r;
            return POLAR_EBUSY;
        }
        r->ticket = s->next_ticket++;
        r->t_submit = now_us();
        s->reqs[r->ticket] = r;
        s->pending.push_back(r);
        *ticket = r->ticket;
    }
    s->cv.notify_all();
    return POLAR_OK;
}

int polar_server_poll(polar_server_t *s, uint64_t ticket, uint8_t *bits_host, float *pm_host, uint8_t *ok_host,
                      int *done) {
    if (!s || !done) return POLAR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return POLAR_EINVAL;
    SrvReq *r = it->second;
    if (!r->done) {
        *done = 0;
        return s->error;
    }
    if (bits_host) std::memcpy(bits_host, r->bits.data(), r->bits.size());
    if (pm_host) std::memcpy(pm_host, r->pm.data(), r->pm.size() * sizeof(float));
    if (ok_host) std::memcpy(ok_host, r->ok.data(), r->ok.size());
    delete r;
    s->reqs.erase(it);
    *done = 1;
    return POLAR_OK;
}

int polar_server_wait(polar_server_t *s, uint64_t ticket, uint32_t timeout_ms) {
    if (!s) return POLAR_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return POLAR_EINVAL;
    SrvReq *r = it->second;
    const bool ok = s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                   [&] { return r->done || s->error != POLAR_OK; });
    if (s->error != POLAR_OK) return s->error;
    return ok ? POLAR_OK : POLAR_ETIMEDOUT;
}

int polar_server_pause(polar_server_t *s, int paused) {
    if (!s) return POLAR_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->paused = paused != 0;
    }
    s->cv.notify_all();
    return POLAR_OK;
}

int polar_server_stats(polar_server_t *s, polar_server_stats_t *out, int reset) {
    if (!s || !out) return POLAR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = s->lat_us.size();
    out->frames = s->frames_done;
    out->info_bits = s->bits_done;
    out->pending = s->pending.size();
    out->admitted = s->admitted.size();
    for (int i = 0; i < kSrvStreams; ++i) out->batches_in_flight += s->busy[i] ? 1u : 0u;
    out->batches = s->batches;
    out->max_batches_in_flight = s->max_inflight;
    if (!s->lat_us.empty()) {
        std::vector<double> v = s->lat_us;
        std::sort(v.begin(), v.end());
        auto q = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
        out->p50_us = q(0.50);
        out->p99_us = q(0.99);
        out->max_us = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_us = sum / v.size();
        out->span_us = s->t_last - s->t_first;
    }
    if (reset) {
        s->lat_us.clear();
        s->lat_frames.clear();
        s->frames_done = s->bits_done = s->batches = s->max_inflight = 0;
        s->t_first = s->t_last = 0.0;
    }
    return s->error;
}

int polar_server_latency(polar_server_t *s, uint32_t min_frames, uint32_t max_frames, double *p50_us,
                         double *p99_us, uint64_t *count) {
    if (!s || min_frames > max_frames) return POLAR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<double> v;
    for (size_t i = 0; i < s->lat_us.size(); ++i)
        if (s->lat_frames[i] >= min_frames && s->lat_frames[i] <= max_frames) v.push_back(s->lat_us[i]);
    std::sort(v.begin(), v.end());
    auto q = [&](double p) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
    if (p50_us) *p50_us = q(0.50);
    if (p99_us) *p99_us = q(0.99);
    if (count) *count = v.size();
    return POLAR_OK;
}

}  // extern "C"
