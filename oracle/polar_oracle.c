/*
 * polar_oracle.c -- CPU oracle for list-CRC decoding of polar codes.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, deliberately
 * unoptimised restatement of "Fast List Decoders for Polar Codes" (Sarkis,
 * Giard, Vardy, Thibeault, Gross) that the CUDA decoder is checked against.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg load
 * it; the product decoder never calls it and shares no code with it.
 *
 * What it computes
 * ----------------
 * Two decoders over one depth-first traversal of the SC decoding tree:
 *
 *   mode OR_BITWISE  -- the LLR SC-list decoder: every leaf has length one
 *                       (Sec. II-B, Eq. (6): the path metric is updated on
 *                       frozen and information bits alike);
 *   mode OR_SPC4     -- the paper's list decoder over the Fast-SSC tree with
 *                       Rate-0, Rate-1, repetition and SPC nodes, SPC nodes of
 *                       length <= 4 ("Dec-SPC-4", Sec. II-D, III, VI);
 *   mode OR_SPC_ANY  -- the same with SPC nodes of any length ("Dec-SPC-4+").
 *
 * Any mode may be or-ed with OR_SYSTEMATIC: the code is systematic (the
 * encoder cited in Sec. I puts payload and CRC in the codeword x itself), so
 * the final pick reads the information bits from x instead of u = x G_N.
 * OR_SPC_ALL_CANDIDATES (tests only) generates all eight SPC candidates even
 * at L = 2; the tests use it to pin the two-candidate rule of R6.
 *
 * Inner nodes apply F (Eq. (1), min-sum), G (Eq. (2)) and Combine (Eq. (3))
 * to every path independently (Sec. III). Leaves generate candidates from
 * the codeword metric of Eq. (9) (Sec. III-A) with the node rules of
 * Sec. III-B (Rate-0), III-C (Rate-1, two least reliable bits), III-D (SPC,
 * four least reliable bits) and III-E (repetition). After every forking leaf
 * the L best candidates survive (Algorithm 1), each with a FULL copy of its
 * parent's state (no sharing). At the end the path with the best metric
 * among those that pass the CRC is the output (Sec. II-B).
 *
 * Metric sign: the paper's PM is <= 0 and larger is better. This file keeps
 * the penalty P = -PM >= 0 (smaller is better) and picks winners by argmin.
 *
 * Readings taken where the paper is silent, ambiguous or garbled:
 *  R1  Rate-0 penalty is sum |min(a,0)| (Eq. (10) and Listing 3); the
 *      alternative form Eq. (11) with max() contradicts both and is garbled.
 *  R2  G is b + (1 - 2 beta) a (Eq. (2)).
 *  R3  h(a) = 1 iff a < 0, so +0 and -0 both decide 0 (Eq. (4)).
 *  R4  Algorithm 1 keeps the exact L best candidates. Ties are broken by
 *      the key (penalty, source slot, candidate index); survivors take new
 *      slots 0.. in ascending (source slot, candidate index) order.
 *  R5  Least reliable bits are ranked by (|a| ascending, index ascending).
 *  R6  SPC candidates are ML xor T for T in the order {}, {1,2}, {1,3},
 *      {1,4}, {2,3}, {2,4}, {3,4}, {1,2,3,4} (ranks of the four least
 *      reliable bits), where ML = HD when the parity of HD is even and
 *      HD xor {1} otherwise. Each penalty is Eq. (9) evaluated directly:
 *      the sum of |a| over the positions where the candidate differs from
 *      HD. (The expanded metrics printed in Sec. III-D agree for even parity
 *      and give odd-weight words for odd parity.) With L = 2 only the first
 *      two candidates are generated (Sec. III-D). They are each source's two
 *      best under the key of R4, so the L = 2 survivors equal those of all
 *      eight (pinned against OR_SPC_ALL_CANDIDATES).
 *  R7  Repetition: the ML candidate (listed first) is all-zero when
 *      P0 <= P1, else all-one (Eq. (5) with the tie to 0).
 *  R8  Float sums: a penalty increment made of least-reliable-bit terms is
 *      accumulated left to right in rank order; a sum over all N_v inputs
 *      (Rate-0, repetition) is the pairwise tree s[i] = x[i] + x[i + n/2]
 *      applied until one value is left. The new penalty is old + increment.
 *  R9  int8 LLRs: F exact, G saturated to [-127, 127], penalties are exact
 *      integers (carried here in float, exact below 2^24). An input of -128
 *      is read as -127 so that every value has a representable negation.
 *  R10 CRC: MSB-first division, register starts at 0, no reflection, no
 *      final xor, over the payload bits in ascending information index; the
 *      CRC occupies the last crc_len information positions.
 *  R11 Final pick: among final paths whose CRC matches, the least
 *      (penalty, slot); when none matches, the least (penalty, slot) with
 *      crc_ok = 0.
 *  R12 Node classification, top down, first match wins: all frozen ->
 *      Rate-0; none frozen -> Rate-1; only the last bit information
 *      (N_v >= 2) -> repetition; only the first bit frozen (N_v >= 4, and
 *      N_v <= 4 in mode OR_SPC4) -> SPC; otherwise split (Sec. II-D). In
 *      mode OR_BITWISE every node longer than one bit is split.
 *
 * Pins: every mode is checked by the tests against brute-force ML, noiseless
 * frames, a textbook SC decoder, the Fig. 1 / Listing 2 example and FER
 * agreement between modes. The final pick (R11) is recomputed outside this
 * file from the final list on frames where a lower-penalty path fails the
 * CRC; int8 saturation (R9) against a hand-worked (4,2) example; pruned
 * selection (R4) against an independent bit-by-bit SC-list written in
 * Python. SPC nodes longer than four bits (mode OR_SPC_ANY)
 * are not exhaustive, so brute-force ML does not fix them; their candidate
 * lists are pinned instead against an independent Chase-II enumeration (all
 * flips of the four least reliable bits, even weight).
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fPIC -shared -pthread.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

#define OR_F32 0
#define OR_I8 1

#define OR_SPC4 0
#define OR_SPC_ANY 1
#define OR_BITWISE 2
#define OR_SYSTEMATIC 0x100
#define OR_SPC_ALL_CANDIDATES 0x200   /* test only: all eight SPC candidates even at L = 2 */

#define NODE_INNER 0
#define NODE_RATE0 1
#define NODE_RATE1 2
#define NODE_REP 3
#define NODE_SPC 4

typedef struct {
    int N, n, K, L, dtype, crc_len, mode, systematic, spc_all, bad_flags;
    uint64_t crc_poly;
    const uint8_t *frozen; /* N bytes, 1 = frozen */
} ocode_t;

/* One decoding path: its own copy of everything. */
typedef struct {
    float *alpha;   /* 2N floats: stage j occupies [2^j, 2^(j+1)), stage n = channel */
    uint8_t *beta;  /* N bits (one per byte): node beta written at its u-range */
    float pen;      /* penalty = -PM */
} opath_t;

typedef struct {
    const ocode_t *c;
    opath_t *paths;  /* active paths, slots 0..na-1 */
    int na;
    opath_t *spare;  /* scratch for the next list */
} olist_t;

/* ---------------- elementary operations (Sec. II-A) ---------------- */

static int h_of(float a) { return a < 0.0f ? 1 : 0; }                 /* Eq. (4), R3 */

static float op_f(float a, float b) {                                  /* Eq. (1), min-sum */
    float ma = fabsf(a), mb = fabsf(b);
    float m = ma < mb ? ma : mb;
    return ((a < 0.0f) != (b < 0.0f)) ? -m : m;
}

static float op_g(float a, float b, int beta, int sat) {               /* Eq. (2), R2, R9 */
    float r = beta ? b - a : b + a;
    if (sat) {
        if (r > 127.0f) r = 127.0f;
        if (r < -127.0f) r = -127.0f;
    }
    return r;
}

/* Pairwise tree sum s[i] = x[i] + x[i + n/2], repeated (R8). x is clobbered. */
static float tree_sum(float *x, int n) {
    while (n > 1) {
        int h = n / 2;
        for (int i = 0; i < h; ++i) x[i] = x[i] + x[i + h];
        n = h;
    }
    return x[0];
}

static float *A(opath_t *p, int j) { return p->alpha + (1 << j); }

/* ---------------- node classification (Sec. II-D, R12) ---------------- */

static int classify(const ocode_t *c, int j, int start) {
    int nv = 1 << j, nf = 0;
    for (int i = 0; i < nv; ++i) nf += c->frozen[start + i] ? 1 : 0;
    if (c->mode == OR_BITWISE && nv > 1) return NODE_INNER;
    if (nf == nv) return NODE_RATE0;
    if (nf == 0) return NODE_RATE1;
    if (nv >= 2 && nf == nv - 1 && !c->frozen[start + nv - 1]) return NODE_REP;
    if (nv >= 4 && nf == 1 && c->frozen[start] &&
        (c->mode == OR_SPC_ANY || nv <= 4)) return NODE_SPC;
    return NODE_INNER;
}

/* ---------------- path storage ---------------- */

static void path_alloc(opath_t *p, int N) {
    p->alpha = (float *)calloc((size_t)2 * N, sizeof(float));
    p->beta = (uint8_t *)calloc((size_t)N, 1);
    p->pen = 0.0f;
}

static void path_free(opath_t *p) {
    free(p->alpha);
    free(p->beta);
}

static void path_copy(opath_t *dst, const opath_t *src, int N) {
    memcpy(dst->alpha, src->alpha, sizeof(float) * 2 * (size_t)N);
    memcpy(dst->beta, src->beta, (size_t)N);
    dst->pen = src->pen;
}

/* ---------------- candidates (Sec. III) ---------------- */

typedef struct {
    int s, c;      /* source slot, candidate index */
    float pen;     /* new penalty */
    /* how to build beta from the source's alpha: */
    int kind;      /* 0: HD xor flips; 1: all zero; 2: all one */
    int nflip;
    int flip[4];   /* positions flipped relative to HD */
} ocand_t;

static int cand_cmp(const void *a, const void *b) {   /* key (pen, s, c), R4 */
    const ocand_t *x = (const ocand_t *)a, *y = (const ocand_t *)b;
    if (x->pen < y->pen) return -1;
    if (x->pen > y->pen) return 1;
    if (x->s != y->s) return x->s < y->s ? -1 : 1;
    if (x->c != y->c) return x->c < y->c ? -1 : 1;
    return 0;
}

/* Rank positions by (|a| ascending, index ascending) and return the first k (R5). */
static void least_reliable(const float *a, int nv, int k, int *m) {
    int *taken = (int *)calloc((size_t)nv, sizeof(int));
    for (int r = 0; r < k; ++r) {
        int best = -1;
        for (int i = 0; i < nv; ++i) {
            if (taken[i]) continue;
            if (best < 0 || fabsf(a[i]) < fabsf(a[best])) best = i;
        }
        m[r] = best;
        taken[best] = 1;
    }
    free(taken);
}

/* Append the candidates of one source path. Returns how many were added. */
static int gen_candidates(const ocode_t *c, int type, const float *a, int nv, int s, float pen_s,
                          ocand_t *out) {
    int cnt = 0;
    if (type == NODE_RATE1) {                                            /* Sec. III-C */
        int m[2] = {0, 0};
        int k = nv >= 2 ? 2 : 1;
        least_reliable(a, nv, k, m);
        float a1 = fabsf(a[m[0]]);
        ocand_t c0 = {s, 0, pen_s, 0, 0, {0, 0, 0, 0}};
        out[cnt++] = c0;
        ocand_t c1 = {s, 1, pen_s + a1, 0, 1, {m[0], 0, 0, 0}};
        out[cnt++] = c1;
        if (nv >= 2) {
            float a2 = fabsf(a[m[1]]);
            ocand_t c2 = {s, 2, pen_s + a2, 0, 1, {m[1], 0, 0, 0}};
            out[cnt++] = c2;
            ocand_t c3 = {s, 3, pen_s + (a1 + a2), 0, 2, {m[0], m[1], 0, 0}};
            out[cnt++] = c3;
        }
    } else if (type == NODE_REP) {                                       /* Sec. III-E */
        float *t0 = (float *)malloc(sizeof(float) * nv);
        float *t1 = (float *)malloc(sizeof(float) * nv);
        for (int i = 0; i < nv; ++i) {
            t0[i] = a[i] < 0.0f ? -a[i] : 0.0f;   /* |min(a,0)|: penalty of all-zero */
            t1[i] = a[i] > 0.0f ? a[i] : 0.0f;    /* |max(a,0)|: penalty of all-one  */
        }
        float p0 = tree_sum(t0, nv), p1 = tree_sum(t1, nv);
        free(t0);
        free(t1);
        ocand_t z = {s, 0, pen_s + p0, 1, 0, {0, 0, 0, 0}};
        ocand_t o = {s, 0, pen_s + p1, 2, 0, {0, 0, 0, 0}};
        if (p0 <= p1) { z.c = 0; o.c = 1; out[cnt++] = z; out[cnt++] = o; }   /* R7 */
        else          { o.c = 0; z.c = 1; out[cnt++] = o; out[cnt++] = z; }
    } else if (type == NODE_SPC) {                                       /* Sec. III-D, R6 */
        static const int T[8][4] = {{0, 0, 0, 0}, {1, 1, 0, 0}, {1, 0, 1, 0}, {1, 0, 0, 1},
                                    {0, 1, 1, 0}, {0, 1, 0, 1}, {0, 0, 1, 1}, {1, 1, 1, 1}};
        int m[4];
        least_reliable(a, nv, 4, m);
        int parity = 0;
        for (int i = 0; i < nv; ++i) parity ^= h_of(a[i]);
        int q = parity == 0;                      /* q = 1 when the parity check holds */
        int ncand = (c->L == 2 && !c->spc_all) ? 2 : 8;
        for (int t = 0; t < ncand; ++t) {
            /* positions differing from HD: T, symmetric-difference {rank 1} when q = 0 */
            int diff[4];
            for (int r = 0; r < 4; ++r) diff[r] = T[t][r];
            if (!q) diff[0] ^= 1;
            float inc = 0.0f;
            int first = 1;
            ocand_t cd = {s, t, 0.0f, 0, 0, {0, 0, 0, 0}};
            for (int r = 0; r < 4; ++r) {
                if (!diff[r]) continue;
                float v = fabsf(a[m[r]]);
                inc = first ? v : inc + v;
                first = 0;
                cd.flip[cd.nflip++] = m[r];
            }
            cd.pen = pen_s + inc;
            out[cnt++] = cd;
        }
    }
    return cnt;
}

static void write_candidate_beta(const ocand_t *cd, const float *a, int nv, uint8_t *dst) {
    if (cd->kind == 1) { memset(dst, 0, (size_t)nv); return; }
    if (cd->kind == 2) { memset(dst, 1, (size_t)nv); return; }
    for (int i = 0; i < nv; ++i) dst[i] = (uint8_t)h_of(a[i]);
    for (int f = 0; f < cd->nflip; ++f) dst[cd->flip[f]] ^= 1;
}

/* ---------------- leaves ---------------- */

static void leaf(olist_t *ls, int type, int j, int start) {
    const ocode_t *c = ls->c;
    int nv = 1 << j;
    if (type == NODE_RATE0) {                                            /* Sec. III-B, R1 */
        float *t = (float *)malloc(sizeof(float) * nv);
        for (int p = 0; p < ls->na; ++p) {
            const float *a = A(&ls->paths[p], j);
            for (int i = 0; i < nv; ++i) t[i] = a[i] < 0.0f ? -a[i] : 0.0f;
            ls->paths[p].pen = ls->paths[p].pen + tree_sum(t, nv);
            memset(ls->paths[p].beta + start, 0, (size_t)nv);
        }
        free(t);
        return;
    }
    /* First pass: all candidates of all sources (Algorithm 1). */
    ocand_t *cand = (ocand_t *)malloc(sizeof(ocand_t) * 8 * (size_t)ls->na);
    int nc = 0;
    for (int s = 0; s < ls->na; ++s)
        nc += gen_candidates(c, type, A(&ls->paths[s], j), nv, s, ls->paths[s].pen, cand + nc);
    /* Second pass: keep the L best (R4). */
    int keep = nc < c->L ? nc : c->L;
    ocand_t *sorted = (ocand_t *)malloc(sizeof(ocand_t) * (size_t)nc);
    memcpy(sorted, cand, sizeof(ocand_t) * (size_t)nc);
    qsort(sorted, (size_t)nc, sizeof(ocand_t), cand_cmp);
    uint8_t *survive = (uint8_t *)calloc((size_t)nc, 1);
    for (int r = 0; r < keep; ++r) {
        for (int i = 0; i < nc; ++i)
            if (cand[i].s == sorted[r].s && cand[i].c == sorted[r].c) { survive[i] = 1; break; }
    }
    /* Survivors, in (source, candidate) order, take slots 0..keep-1 with full copies. */
    int slot = 0;
    for (int i = 0; i < nc; ++i) {
        if (!survive[i]) continue;
        opath_t *dst = &ls->spare[slot++];
        const opath_t *src = &ls->paths[cand[i].s];
        path_copy(dst, src, c->N);
        dst->pen = cand[i].pen;
        write_candidate_beta(&cand[i], A((opath_t *)src, j), nv, dst->beta + start);
    }
    opath_t *tmp = ls->paths;
    ls->paths = ls->spare;
    ls->spare = tmp;
    ls->na = keep;
    free(cand);
    free(sorted);
    free(survive);
}

/* ---------------- depth-first traversal (Sec. II-A, II-D, III) ---------------- */

static void decode_node(olist_t *ls, int j, int start) {
    int type = classify(ls->c, j, start);
    if (type != NODE_INNER) { leaf(ls, type, j, start); return; }
    int h = 1 << (j - 1);
    int sat = ls->c->dtype == OR_I8;
    for (int p = 0; p < ls->na; ++p) {                                   /* F, Eq. (1) */
        float *in = A(&ls->paths[p], j), *out = A(&ls->paths[p], j - 1);
        for (int i = 0; i < h; ++i) out[i] = op_f(in[i], in[i + h]);
    }
    decode_node(ls, j - 1, start);
    for (int p = 0; p < ls->na; ++p) {                                   /* G, Eq. (2) */
        float *in = A(&ls->paths[p], j), *out = A(&ls->paths[p], j - 1);
        const uint8_t *bl = ls->paths[p].beta + start;
        for (int i = 0; i < h; ++i) out[i] = op_g(in[i], in[i + h], bl[i], sat);
    }
    decode_node(ls, j - 1, start + h);
    for (int p = 0; p < ls->na; ++p) {                                   /* Combine, Eq. (3) */
        uint8_t *b = ls->paths[p].beta + start;
        for (int i = 0; i < h; ++i) b[i] ^= b[i + h];
    }
}

/* ---------------- CRC and encoding ---------------- */

/* CRC register after feeding `nbits` bits MSB-first from `init` (R10). */
uint64_t oracle_crc(const uint8_t *bits, int nbits, uint64_t poly, int clen, uint64_t init) {
    if (clen <= 0) return 0;
    uint64_t mask = clen >= 64 ? ~0ull : ((1ull << clen) - 1);
    uint64_t reg = init & mask;
    for (int t = 0; t < nbits; ++t) {
        uint64_t fb = ((reg >> (clen - 1)) & 1u) ^ (uint64_t)(bits[t] & 1u);
        reg = (reg << 1) & mask;
        if (fb) reg ^= poly & mask;
    }
    return reg;
}

/* x = u G_N (natural order); G_N is an involution. In place. */
void oracle_polar_transform(uint8_t *v, int N) {
    for (int h = 1; h < N; h *= 2)
        for (int i = 0; i < N; ++i)
            if (!(i & h)) v[i] ^= v[i + h];
}

/* ---------------- whole-frame decode ---------------- */

typedef struct {
    float pen;
    int ok;
    int slot;
} opick_t;

/* Run the list decoder on one frame. On return ls holds the final list. */
static void run_list(olist_t *ls, const ocode_t *c, const void *llr) {
    ls->c = c;
    ls->na = 1;
    opath_t *p0 = &ls->paths[0];
    float *ch = A(p0, c->n);
    if (c->dtype == OR_I8) {
        const int8_t *q = (const int8_t *)llr;
        for (int i = 0; i < c->N; ++i) ch[i] = q[i] < -127 ? -127.0f : (float)q[i];  /* R9 */
    } else {
        memcpy(ch, llr, sizeof(float) * c->N);
    }
    p0->pen = 0.0f;
    memset(p0->beta, 0, (size_t)c->N);
    decode_node(ls, c->n, 0);
}

static void list_init(olist_t *ls, const ocode_t *c) {
    ls->paths = (opath_t *)calloc((size_t)c->L, sizeof(opath_t));
    ls->spare = (opath_t *)calloc((size_t)c->L, sizeof(opath_t));
    for (int i = 0; i < c->L; ++i) {
        path_alloc(&ls->paths[i], c->N);
        path_alloc(&ls->spare[i], c->N);
    }
}

static void list_free(olist_t *ls, const ocode_t *c) {
    for (int i = 0; i < c->L; ++i) {
        path_free(&ls->paths[i]);
        path_free(&ls->spare[i]);
    }
    free(ls->paths);
    free(ls->spare);
}

/* Final pick (Sec. II-B, R10, R11). Writes the payload bits of the winner.
 * The information bits are those of u = x G_N, or of x for a systematic code. */
static opick_t final_pick(const olist_t *ls, const ocode_t *c, uint8_t *payload_bits) {
    int N = c->N, k = c->K - c->crc_len;
    uint8_t *u = (uint8_t *)malloc((size_t)N);
    uint8_t *info = (uint8_t *)malloc((size_t)(c->K > 0 ? c->K : 1));
    opick_t best = {0.0f, 0, -1};
    for (int p = 0; p < ls->na; ++p) {
        memcpy(u, ls->paths[p].beta, (size_t)N);
        if (!c->systematic) oracle_polar_transform(u, N);
        int t = 0;
        for (int i = 0; i < N; ++i) if (!c->frozen[i]) info[t++] = u[i];
        int ok = 1;
        if (c->crc_len > 0) {
            uint64_t r = oracle_crc(info, k, c->crc_poly, c->crc_len, 0);
            for (int b = 0; b < c->crc_len; ++b)
                if ((int)((r >> (c->crc_len - 1 - b)) & 1u) != info[k + b]) ok = 0;
        }
        float pen = ls->paths[p].pen;
        int better;
        if (best.slot < 0) better = 1;
        else if (ok != best.ok) better = ok > best.ok;
        else better = pen < best.pen;   /* equal penalty keeps the lower slot */
        if (better) { best.pen = pen; best.ok = ok; best.slot = p; }
    }
    memcpy(u, ls->paths[best.slot].beta, (size_t)N);
    if (!c->systematic) oracle_polar_transform(u, N);
    int t = 0;
    for (int i = 0; i < N && t < k; ++i) if (!c->frozen[i]) payload_bits[t++] = u[i];
    free(u);
    free(info);
    return best;
}

static int check_code(const ocode_t *c) {
    if (c->N < 2 || (c->N & (c->N - 1)) || c->N > 65536) return -1;
    if (c->L < 1 || c->L > 1024) return -1;
    if (c->crc_len < 0 || c->crc_len > 63 || c->crc_len > c->K) return -1;
    if (c->dtype != OR_F32 && c->dtype != OR_I8) return -1;
    if (c->mode < 0 || c->mode > 2 || c->bad_flags) return -1;
    return 0;
}

static void fill_code(ocode_t *c, int N, int K, const uint8_t *frozen, int L, int dtype,
                      int crc_len, uint64_t crc_poly, int mode) {
    c->N = N;
    c->n = 0;
    while ((1 << c->n) < N) c->n++;
    c->K = K;
    c->frozen = frozen;
    c->L = L;
    c->dtype = dtype;
    c->crc_len = crc_len;
    c->crc_poly = crc_poly;
    c->mode = mode & 0xFF;
    c->systematic = (mode & OR_SYSTEMATIC) ? 1 : 0;
    c->spc_all = (mode & OR_SPC_ALL_CANDIDATES) ? 1 : 0;
    c->bad_flags = (mode & ~(0xFF | OR_SYSTEMATIC | OR_SPC_ALL_CANDIDATES)) != 0;
}

/* ---------------- exported entry points ---------------- */

/* Decode one frame and return the final list: words[L*N] (codewords, one bit
 * per byte), pens[L], *n_final. Returns 0 or -1 on bad arguments. */
int oracle_decode_list(int N, int K, const uint8_t *frozen, int L, int dtype, int mode,
                       const void *llr, uint8_t *words, float *pens, int *n_final) {
    ocode_t c;
    fill_code(&c, N, K, frozen, L, dtype, 0, 0, mode);
    if (check_code(&c)) return -1;
    olist_t ls;
    list_init(&ls, &c);
    run_list(&ls, &c, llr);
    for (int p = 0; p < ls.na; ++p) {
        memcpy(words + (size_t)p * N, ls.paths[p].beta, (size_t)N);
        pens[p] = ls.paths[p].pen;
    }
    *n_final = ls.na;
    list_free(&ls, &c);
    return 0;
}

typedef struct {
    const ocode_t *c;
    const uint8_t *llr;
    size_t llr_stride;
    int n_frames, tid, nthreads;
    uint8_t *bits;
    float *pm;
    uint8_t *ok;
    int32_t *slot;
} ojob_t;

static void *worker(void *arg) {
    ojob_t *jb = (ojob_t *)arg;
    const ocode_t *c = jb->c;
    int k = c->K - c->crc_len;
    int kb = (k + 7) / 8;
    olist_t ls;
    list_init(&ls, c);
    uint8_t *pl = (uint8_t *)malloc((size_t)(k > 0 ? k : 1));
    for (int f = jb->tid; f < jb->n_frames; f += jb->nthreads) {
        run_list(&ls, c, jb->llr + (size_t)f * jb->llr_stride);
        opick_t pk = final_pick(&ls, c, pl);
        uint8_t *dst = jb->bits + (size_t)f * kb;
        memset(dst, 0, (size_t)kb);
        for (int b = 0; b < k; ++b) dst[b / 8] |= (uint8_t)(pl[b] << (b % 8));  /* LSB-first */
        jb->pm[f] = pk.pen;
        if (jb->ok) jb->ok[f] = (uint8_t)pk.ok;
        if (jb->slot) jb->slot[f] = pk.slot;
    }
    free(pl);
    list_free(&ls, c);
    return NULL;
}

/* Decode n_frames frames. llr is [n_frames][N] float32 (dtype 0) or int8
 * (dtype 1). bits is [n_frames][ceil(k/8)] (payload, LSB-first), pm the
 * winning penalty, ok the CRC flag, slot the winning slot (ok/slot may be
 * NULL). Frames are spread over n_threads POSIX threads. */
int oracle_decode(int N, int K, const uint8_t *frozen, int L, int dtype, int mode, int crc_len,
                  uint64_t crc_poly, const void *llr, int n_frames, uint8_t *bits, float *pm,
                  uint8_t *ok, int32_t *slot, int n_threads) {
    ocode_t c;
    fill_code(&c, N, K, frozen, L, dtype, crc_len, crc_poly, mode);
    if (check_code(&c) || n_frames < 0) return -1;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > n_frames) n_threads = n_frames > 0 ? n_frames : 1;
    size_t esz = dtype == OR_I8 ? 1 : 4;
    ojob_t *jobs = (ojob_t *)calloc((size_t)n_threads, sizeof(ojob_t));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    for (int t = 0; t < n_threads; ++t) {
        ojob_t j = {&c, (const uint8_t *)llr, esz * N, n_frames, t, n_threads, bits, pm, ok, slot};
        jobs[t] = j;
    }
    if (n_threads == 1) {
        worker(&jobs[0]);
    } else {
        for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, worker, &jobs[t]);
        for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    }
    free(jobs);
    free(th);
    return 0;
}

/* The decoding schedule of the tree, as the unrolled operation list of
 * Listing 2: one entry per F, G, Combine or leaf, in execution order.
 * ops[3*i] = kind (0 F, 1 G, 2 Combine, 10 + node type for a leaf),
 * ops[3*i+1] = N_v of the node, ops[3*i+2] = first u index of the node.
 * Returns the number of entries (or -1 if cap is too small). */
static int sched_rec(const ocode_t *c, int j, int start, int *ops, int cap, int cnt) {
    if (cnt < 0) return cnt;
    int type = classify(c, j, start);
    int nv = 1 << j;
    if (type != NODE_INNER) {
        if (cnt >= cap) return -1;
        ops[3 * cnt] = 10 + type; ops[3 * cnt + 1] = nv; ops[3 * cnt + 2] = start;
        return cnt + 1;
    }
    if (cnt >= cap) return -1;
    ops[3 * cnt] = 0; ops[3 * cnt + 1] = nv; ops[3 * cnt + 2] = start;
    cnt = sched_rec(c, j - 1, start, ops, cap, cnt + 1);
    if (cnt < 0 || cnt >= cap) return -1;
    ops[3 * cnt] = 1; ops[3 * cnt + 1] = nv; ops[3 * cnt + 2] = start;
    cnt = sched_rec(c, j - 1, start + nv / 2, ops, cap, cnt + 1);
    if (cnt < 0 || cnt >= cap) return -1;
    ops[3 * cnt] = 2; ops[3 * cnt + 1] = nv; ops[3 * cnt + 2] = start;
    return cnt + 1;
}

int oracle_schedule(int N, const uint8_t *frozen, int mode, int *ops, int cap) {
    ocode_t c;
    fill_code(&c, N, 0, frozen, 1, OR_F32, 0, 0, mode);
    if (check_code(&c)) return -1;
    return sched_rec(&c, c.n, 0, ops, cap, 0);
}
