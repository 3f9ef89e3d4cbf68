// polar_internal.h -- shared between the host runtime (polar_capi.cu) and the
// decode kernels (polar_kernels.cu). Not part of the public ABI.
#pragma once

#include <stdint.h>
#include <cuda_runtime.h>

namespace polar {

constexpr int kMaxLogN = 12;   // N <= 4096
constexpr int kMaxL = 32;      // narrow kernels: one warp lane per path
constexpr int kMaxWideL = 128; // wide kernel: one CTA thread per path

// Operation kinds of the unrolled schedule (Listing 2 of the paper).
enum OpKind : uint32_t {
    OP_F = 0,      // alpha_l = F(alpha_v)                      Eq. (1)
    OP_G = 1,      // alpha_r = G(alpha_v, beta_l)              Eq. (2)
    OP_COMB = 2,   // beta_v = [beta_l ^ beta_r, beta_r]        Eq. (3)
    OP_R0 = 3,     // Rate-0 leaf                               Sec. III-B
    OP_R1 = 4,     // Rate-1 leaf                               Sec. III-C
    OP_REP = 5,    // repetition leaf                           Sec. III-E
    OP_SPC = 6,    // single-parity-check leaf                  Sec. III-D
    OP_SUB = 7     // a whole subtree of <= 2^kSubLog bits in registers
};

// Subtrees rooted at this stage or below run as one OP_SUB operation: warp 0,
// one lane per path, LLRs / beta / penalty in registers. An OP_SUB at stage
// kSubLog + 1 is an inner node whose two children are such subtrees: F, left
// subtree, G, right subtree and Combine in one operation (its descriptor index
// names the left subtree's descriptor; the right one follows it).
constexpr int kSubLog = 4;

// One schedule entry: kind | stage j << 4 | dest << 8 | solo << 9 | sync << 10.
//   j     stage of the node (N_v = 2^j)
//   dest  where the node's beta goes: 0 = left-child buffer BL[j],
//         1 = right-child / root buffer BR
//   solo  warp 0 of the frame's group runs the operation alone
//   sync  a group barrier follows (else only warp 0 synchronises)
__host__ __device__ inline uint32_t op_make(uint32_t kind, uint32_t j, uint32_t dest) {
    return kind | (j << 4) | (dest << 8);
}
__host__ __device__ inline uint32_t op_kind(uint32_t op) { return op & 15u; }
__host__ __device__ inline int op_stage(uint32_t op) { return (int)((op >> 4) & 15u); }
__host__ __device__ inline int op_dest(uint32_t op) { return (int)((op >> 8) & 1u); }
__host__ __device__ inline bool op_solo(uint32_t op) { return ((op >> 9) & 1u) != 0; }
__host__ __device__ inline bool op_sync(uint32_t op) { return ((op >> 10) & 1u) != 0; }
constexpr uint32_t OP_SOLO = 1u << 9;
constexpr uint32_t OP_SYNC = 1u << 10;
// OP_F / OP_G only: bits 16..27 = first bit index s of the node. The node at
// stage j' >= j containing bit s is the right child of its parent iff bit j'
// of s is set; stages evaluated from the channel (Layout::virt_mask) need it.
__host__ __device__ inline uint32_t op_with_start(uint32_t op, uint32_t s) { return op | (s << 16); }
__host__ __device__ inline uint32_t op_start(uint32_t op) { return (op >> 16) & 0xFFFu; }
// OP_SUB only: bit 11 = the subtree forks paths, bits 12..14 = log2 of the
// product of its leaves' candidate counts (saturated at 6; the live paths
// become min(L, L_a * 2^m)), bits 15.. = index of its descriptor.
__host__ __device__ inline bool op_sub_fork(uint32_t op) { return ((op >> 11) & 1u) != 0; }
__host__ __device__ inline int op_sub_logmult(uint32_t op) { return (int)((op >> 12) & 7u); }
__host__ __device__ inline uint32_t op_sub_desc(uint32_t op) { return op >> 15; }
// Subtree descriptor: pre-order node kinds, 3 bits each (0 = inner node,
// OP_R0 .. OP_SPC = leaf), 21 per 64-bit word, two words per subtree.

// Bit-packed beta: words per path for a node of 2^j bits.
__host__ __device__ inline int beta_words(int j) { return j >= 5 ? 1 << (j - 5) : 1; }

// Per-frame memory layout. Byte offsets inside one frame-group's shared
// memory region, or inside its global scratch region for buffers that do not
// fit the shared-memory budget ("spilled"). Alpha and left-beta buffers exist
// only for stages kSubLog..n-1: lower stages live in registers (OP_SUB).
struct Layout {
    uint32_t alpha[kMaxLogN];      // stage j: L rows of 2^j elements
    uint32_t bl[kMaxLogN];         // left-child beta of stage j: L rows of beta_words(j) words
    uint32_t br;                   // right/root beta: L rows of beta_words(n) words
    uint32_t chan;                 // channel LLRs (stage n), N elements
    uint32_t idx[2];               // alpha stage -> physical row, [L][16] bytes, double buffered
    uint32_t bidx[2];              // left-beta stage -> physical row, same shape
    uint32_t pen[2];               // penalties, [L] float or int32, double buffered
    uint32_t surv;                 // survivor keys in new-slot order, L x 8 bytes
    uint32_t ubuf;                 // winner's u vector, beta_words(n) words
    uint32_t bytes;                // shared memory per group (multiple of 16)
    uint32_t spill_mask;           // bit j: alpha stage j in global scratch
    uint32_t bl_spill;             // bit j: left beta of stage j in global scratch
    uint32_t flags;                // bit 0: BR in global scratch, bit 1: channel in global scratch
    uint32_t virt_mask;            // bit j: alpha stage j is not stored; F / G reading it evaluate it
                                   // from the channel (stages n-D .. n-1, every node there inner)
    uint64_t galpha[kMaxLogN];     // global offsets of spilled buffers
    uint64_t gbl[kMaxLogN];
    uint64_t gbr, gchan;
    uint64_t gbytes;               // global scratch per group
};
constexpr uint32_t LAY_BR_GLOBAL = 1u;
constexpr uint32_t LAY_CHAN_GLOBAL = 2u;

// Everything the decoder needs about one code (and one launch shape).
struct CodeView {
    const uint32_t *ops;           // schedule with solo / sync flags
    const uint32_t *syn;           // [N/8][256] CRC syndrome of each codeword byte
    const uint16_t *info;          // [K] information positions, ascending
    const unsigned long long *desc;// subtree descriptors, two words each
    int n_ops;
    int N, n, L, K, k, kb, crc_len;
    int systematic;                // payload read from x, not from u = x G_N
    int pack;                      // 1 only where it applies (L <= 16, one warp per frame): run register
                                   // subtrees 32 / L frames to a warp in lockstep rounds, selection in
                                   // L-lane segments
    Layout lay;
};

struct Params {                    // plain form: one code
    CodeView cv;
    const void *llr;               // [n_frames][N]
    uint8_t *bits;                 // [n_frames][kb]
    float *pm;
    uint8_t *ok;
    int32_t *slot;
    uint32_t n_frames;
    uint8_t *scratch;              // global scratch (spilled stages), lay.gbytes per group
    int groups_per_cta;
    const uint32_t *frame_idx;     // optional: decode only frames frame_idx[0 .. *frame_cnt)
    const uint32_t *frame_cnt;
};

struct BatchItem {                 // one frame of a batched launch
    uint32_t cls;                  // index into the class table
    uint32_t frame;                // output index (pm, ok, slot)
    uint64_t llr_off;              // byte offset of the frame's LLR row
    uint64_t bits_off;             // byte offset of the frame's payload row
};

struct BatchParams {               // batched form: frames of several codes
    const CodeView *classes;
    const BatchItem *items;        // ordered by decreasing cost
    uint32_t n_items;
    uint32_t *counter;             // work counter, zero at launch
    const uint8_t *llr;
    uint8_t *bits;
    float *pm;
    uint8_t *ok;
    int32_t *slot;
    uint8_t *scratch;
    uint64_t gbytes;               // global scratch per group
    uint32_t group_bytes;          // shared memory per group (view + frame region)
    uint32_t view_bytes;           // CodeView copy + work slot, 16-byte aligned
    int groups_per_cta;
};

// Plain-form CTAs hold up to this many threads (frame groups of 1, 2 or 4
// warps); the groups of one CTA decode the same code in lockstep.
constexpr int kMaxCtaThreads = 512;

struct LaunchShape {
    int warps;                     // warps per frame group (1, 2, 4)
    uint32_t budget;               // shared-memory budget per group the layout was built for
    uint32_t *d_ops;               // schedule with this shape's solo / sync flags (device)
    int groups_per_cta;
    int threads;                   // per CTA
    uint32_t smem;                 // dynamic shared memory per CTA
    int pack;                      // CodeView::pack; also picks the kernels that hold the packed code
    Layout lay;
};

// Launch one decode (kernels are instantiated for float / int8 and 1, 2, 4 warps).
cudaError_t launch_decode(int dtype, const LaunchShape &shape, const Params &p, int grid,
                          cudaStream_t stream);
// Resident CTAs per SM for a shape (0 if it cannot launch).
int occupancy(int dtype, const LaunchShape &shape);
// Indices of the frames whose CRC flag is 0 (order unspecified) and their count.
cudaError_t launch_crc_failures(const uint8_t *ok, uint32_t n_frames, uint32_t *idx, uint32_t *cnt,
                                cudaStream_t stream);
// Batched form: CTAs of `threads` threads (groups of `warps` warps) with
// `smem` bytes of shared memory.
cudaError_t launch_batch(int dtype, int warps, bool seg, const BatchParams &b, int grid, uint32_t smem, int threads,
                         cudaStream_t stream);
int occupancy_batch(int dtype, int warps, bool seg, uint32_t smem, int threads);
// Wide lists (L = 64, 128): one CTA of L threads per frame over the fully
// unrolled schedule; every stage in the CTA's global scratch region.
struct WideView {
    const uint32_t *xops;          // fully unrolled schedule (F, G, Combine, leaves)
    const uint32_t *syn;           // [N/8][256] CRC syndrome of each codeword byte
    const uint16_t *info;          // [K] information positions
    int n_xops;
    int N, n, L, K, k, kb, crc_len, systematic;
    // Buffer locations: a global scratch offset, or, with kWideInSmem set, an
    // offset into the CTA's shared memory after its tables.
    uint64_t galpha[kMaxLogN];     // stage j: L rows of 2^j elements
    uint64_t gbl[kMaxLogN];        // left beta of stage j: L rows of beta_words(j) words
    uint64_t gbr, gchan;           // right/root beta, channel row
    uint64_t gbytes;               // global scratch per CTA
    uint32_t sbytes;               // shared memory of the buffers kept on chip
};
constexpr uint64_t kWideInSmem = 1ull << 63;

struct WideParams {
    WideView v;
    const void *llr;
    uint8_t *bits;
    float *pm;
    uint8_t *ok;
    int32_t *slot;
    uint32_t n_frames;
    uint8_t *scratch;              // v.gbytes per CTA
    const uint32_t *frame_idx;     // optional indirection, as in Params
    const uint32_t *frame_cnt;
};

uint32_t wide_smem_bytes(int L, int n);   // the CTA's tables; the launch adds WideView::sbytes
int occupancy_wide(int dtype, int L, uint32_t smem);
cudaError_t launch_wide(int dtype, const WideParams &p, int grid, cudaStream_t stream);

// ---- L = 1 (Fast-SSC): one lane per frame, 32 frames per warp in lockstep ----
constexpr int kSc1Threads = 256;   // CTA size, unless fewer warps' shared memory fits

// Schedule entry of the L = 1 kernel: kind | stage j << 4 | first bit s << 8.
__host__ __device__ inline uint32_t sc1_op(uint32_t kind, uint32_t j, uint32_t s) {
    return kind | (j << 4) | (s << 8);
}

struct Sc1Params {
    const uint32_t *ops;           // sc1_op entries, fully unrolled (F/G/Combine/leaves)
    int n_ops;
    const uint32_t *syn;           // [N/8][256] CRC syndrome of each codeword byte
    const uint16_t *info;          // [K] information positions, ascending
    int n, k, kb, crc_len, systematic;
    int split;                     // alpha stages below it in shared memory, the rest in global scratch
    int beta_smem;                 // beta rows in shared memory (else in global scratch)
    uint32_t warp_bytes, beta_off; // shared memory of one warp (32 frames); offset of its beta rows
    uint64_t warp_gbytes;          // global scratch of one warp
    uint8_t *scratch;              // warp_gbytes per warp of the grid (when split < n)
    int drop;                      // float: drop dead spilled stages from L2 (the DROP instantiation)
    const void *llr;               // [n_frames][N]
    uint8_t *bits;                 // [n_frames][kb]
    float *pm;
    uint8_t *ok;
    int32_t *slot;
    uint32_t n_frames;
    const uint32_t *frame_idx;     // optional indirection, as in Params
    const uint32_t *frame_cnt;
};

// Per-warp shared memory and global scratch of the L = 1 kernel for a budget.
struct Sc1Layout {
    int split, beta_smem;
    uint32_t warp_bytes, beta_off;
    uint64_t warp_gbytes;
};
void sc1_layout(int n, int es, uint32_t budget, Sc1Layout *lay);
int occupancy_sc1(int dtype, uint32_t warp_bytes, int warps, bool drop);
cudaError_t launch_sc1(int dtype, const Sc1Params &p, int grid, int warps, cudaStream_t stream);

// The L = 1 kernel for small batches (polar_sc1w.cu): one warp per frame, the
// lanes over a node's elements, every stored stage in the warp's shared memory.
constexpr int kSc1wThreads = 256;  // most threads per CTA
struct Sc1wParams {
    const uint32_t *ops;           // sc1_op entries, fully unrolled (F/G/Combine/leaves)
    int n_ops;
    const uint32_t *syn;           // [N/8][256] CRC syndrome of each codeword byte
    const uint16_t *info;          // [K] information positions, ascending
    int n, k, kb, crc_len, systematic;
    int root_leaf;                 // the root is a leaf: its input (the channel) is copied to stage n
    int warp_bytes, beta_off;      // shared memory of one warp; offset of its beta row
    const void *llr;               // [n_frames][N]
    uint8_t *bits;                 // [n_frames][kb]
    float *pm;
    uint8_t *ok;
    int32_t *slot;
    uint32_t n_frames;
    const uint32_t *frame_idx;     // optional indirection, as in Params
    const uint32_t *frame_cnt;
};
int sc1w_warp_bytes(int n, int es, bool root_leaf, int *beta_off);
int occupancy_sc1w(int dtype, int n, bool root_leaf, int warps);
cudaError_t launch_sc1w(int dtype, const Sc1wParams &p, int grid, int warps, cudaStream_t stream);

}  // namespace polar
