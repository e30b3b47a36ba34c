/*
 * replay.c -- sequential replay of the kernels' documented reduction order.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The twofold pair (value, error) depends on the order of the additions
 * (Example 1 fixes it for one sequential loop).  The kernels split the input
 * into independent chains and merge the chains' pairs; that order is a fixed,
 * documented function of the launch shape.  This file replays it one
 * operation at a time, so that a kernel's output can be checked bit for bit.
 * It shares no code with the kernels: it is written from the description
 * below, with the per-item steps of Examples 1 and 3 and the merge built on
 * Knuth's TWO-SUM (Theorem 2).
 *
 * Per-item update of a chain (s, e), item y (for a dot, y = p = RN(a*b) and
 * ep = RN(a*b - p) is its exact rounding error; the "literal" dot variants
 * and Kahan take the rounded product alone, ep = 0, as the paper's dot
 * functions do):
 *   plain      s <- s + y
 *   fast       t <- s + y; c <- (t - s) - y; e <- e - c; s <- t     (Ex. 1)
 *              dot: e <- e + (ep - c)
 *   rigorous   t <- s + y; yt <- t - s; dy <- y - yt; ds <- s - (t - yt);
 *              e <- e + (ds + dy); s <- t                            (Ex. 3)
 *              dot: e <- e + ((ds + dy) + ep)
 *   wide       S <- S + y in binary64, y (or the binary64 product of two
 *              binary32 operands, which is exact) widened exactly; for
 *              binary64 data the accumulator is binary128 (the paper's
 *              __float128 'sumd'), y or the binary128 product of two
 *              binary64 operands (exact) added with one binary128 rounding,
 *              chains merged by binary128 additions, output
 *              (RN64(S), RN64(S - RN64(S))).
 *   kahan      Example 2 with e = -c: y' <- y + e; t <- s + y';
 *              e <- y' - (t - s); s <- t   (bit for bit Example 2's
 *              y - c, (t - s) - y' negated, since negation is exact)
 * Merge of two pairs:  (v, q) <- TWO-SUM(v1, v2);  e <- (e1 + e2) + q
 * (twofold and Kahan).  Plain and wide merge by one addition.  Every state
 * starts at (+0, +0).
 * Variant codes: 0 plain, 1 fast, 2 rigorous, 3 wide, 4 kahan, 5 fast and
 * 6 rigorous with the literal (rounded, error-free-less) product.
 *
 * Flat order (one vector x of n elements, launch block B, unroll U, grid G):
 *   V = 16 / sizeof(element); vector j holds elements jV .. jV+V-1.
 *   Thread g = b*B + t (P = G*B threads) takes vectors j = g + P*m,
 *   m = 0, 1, ...; element l of vector j feeds chain c = (m mod U)*V + l of
 *   that thread.  The last, partial vector (n mod V elements) is vector
 *   floor(n/V) and is treated the same way.
 *   Each thread folds its U*V chains as a tree: for w = UV/2, ..., 1:
 *   chain[c] <- merge(chain[c], chain[c + w]) for c < w.
 *   Binary64 twofold variants (fast, rigorous, kahan, the literal dots): the
 *   B thread pairs of a block fold by the same tree: for w = B/2, ..., 1:
 *   pair[t] <- merge(pair[t], pair[t + w]) for t < w; pair 0 is the block's.
 *   The other variants: each warp of 32 threads folds as a butterfly: for
 *   o = 16, 8, 4, 2, 1: pair[i] <- merge(pair[i], pair[i xor o]), lane 0
 *   holding the result; the W = B/32 warp pairs of a block fold by the same
 *   butterfly with o = W/2, ..., 1.
 *   Grid fold of the G block pairs: thread t of one block of B threads starts
 *   from pair t (identity if t >= G) and merges pairs t+B, t+2B, ... in turn;
 *   then the B thread pairs fold as a block's do.  For binary32 data the
 *   grid fold runs in binary64 (the block pairs widen exactly), except for
 *   the plain variant, which stays in binary32 throughout.
 *   Output for binary32 data from the binary64 pair (V, E):
 *   v = RN32(V), e = RN32((V - v) + E) [wide: E = 0]; binary64 data: (V, E).
 *
 * CSR order (segments [off[s], off[s+1]) of one concatenated vector; tile T):
 *   The concatenated vector is cut into tiles of T elements.  A segment's
 *   piece in tile w is the part of the segment that lies in the tile.  In a
 *   piece, element i (r = i - wT within the tile, q = floor(r/V)) goes to
 *   lane q mod 32, chain ((floor(q/32)) mod U)*V + (r mod V).  Lanes fold
 *   their chains by the tree above and the 32 lanes by the butterfly.  A
 *   segment that lies in one tile outputs its piece pair.  A segment over k
 *   tiles merges its k piece pairs (binary64 for binary32 data, except plain):
 *   for k <= 32 as 32 lanes holding pieces 0..k-1 (+0 pairs after them)
 *   folded by the butterfly; for k > 32 by a pairwise tree in tile order:
 *   with w = 1, 2, 4, ..., the pair at piece j (j a multiple of 2w) becomes
 *   merge(pair j, pair j + w) when j + w < k and stays as it is otherwise;
 *   the root is piece 0's pair.  The output rule above applies.  An empty
 *   segment outputs (+0, +0).
 */
#include "oracle.h"
#include "orc_internal.h"
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* arithmetic in the working precision: f32 != 0 means binary32.  Values are
   held in doubles that are always representable in the working precision. */
static inline double ADD(int f32, double a, double b) {
    if (f32) { float r = (float)a + (float)b; return (double)r; }
    return a + b;
}
static inline double SUB(int f32, double a, double b) {
    if (f32) { float r = (float)a - (float)b; return (double)r; }
    return a - b;
}

/* chain state: (s, e) in the working precision, or a binary128 accumulator q */
typedef struct { double s, e; _Float128 q; } pr_t;

static inline void two_sum(int f, double a, double b, double* x, double* y) {
    double xx = ADD(f, a, b);
    double bv = SUB(f, xx, a);
    double av = SUB(f, xx, bv);
    double bs = SUB(f, b, bv);
    double as = SUB(f, a, av);
    *x = xx;
    *y = ADD(f, as, bs);
}

/* merge in working precision f (2: binary128); twofold = 0 for plain/wide (one add) */
static inline pr_t merge(int f, int twofold, pr_t a, pr_t b) {
    pr_t r;
    r.q = 0;
    if (f == 2) { r.s = 0.0; r.e = 0.0; r.q = a.q + b.q; return r; }
    if (!twofold) { r.s = ADD(f, a.s, b.s); r.e = 0.0; return r; }
    double v, q;
    two_sum(f, a.s, b.s, &v, &q);
    r.s = v;
    r.e = ADD(f, ADD(f, a.e, b.e), q);
    return r;
}

typedef struct {
    int dtype, op, variant;
    const void* x; const void* y;
} prob_t;

/* feed element i of the problem into chain st */
static inline void feed(const prob_t* P, pr_t* st, int64_t i) {
    int f = (P->dtype == ORC_F32);
    double y, ep = 0.0;
    if (P->dtype == ORC_F32) {
        float a = ((const float*)P->x)[i];
        if (P->op == 0) { y = a; }
        else {
            float b = ((const float*)P->y)[i];
            if (P->variant == 3) { y = (double)a * (double)b; }           /* exact */
            else if (P->variant == 0 || P->variant >= 4) { float pp = a * b; y = pp; }
            else { float pp, ee; orc_two_product_f32(&a, &b, 1, &pp, &ee); y = pp; ep = ee; }
        }
    } else {
        double a = ((const double*)P->x)[i];
        if (P->op == 0) { y = a; }
        else {
            double b = ((const double*)P->y)[i];
            if (P->variant == 0 || P->variant >= 4) { y = a * b; }
            else { double pp, ee; orc_two_product_f64(&a, &b, 1, &pp, &ee); y = pp; ep = ee; }
        }
    }
    int v = P->variant == 5 ? 1 : (P->variant == 6 ? 2 : P->variant);
    if (P->dtype == ORC_F64 && P->variant == 3) {          /* binary128 accumulator */
        const double a = ((const double*)P->x)[i];
        if (P->op == 0) st->q = st->q + (_Float128)a;
        else st->q = st->q + (_Float128)a * (_Float128)((const double*)P->y)[i];
        return;
    }
    switch (v) {
    case 0:  /* plain */
        st->s = ADD(f, st->s, y);
        break;
    case 3:  /* wide: binary64 accumulator */
        st->s = st->s + y;
        break;
    case 1: { /* fast, Example 1: Dekker's correction c of s + y, subtracted from e */
        const double x = ADD(f, st->s, y);
        const double c = SUB(f, SUB(f, x, st->s), y);
        st->e = (P->op == 0) ? SUB(f, st->e, c) : ADD(f, st->e, SUB(f, ep, c));
        st->s = x;
        break; }
    case 4: { /* kahan, Example 2 with e = -c */
        double yk = ADD(f, y, st->e);
        double t = ADD(f, st->s, yk);
        st->e = SUB(f, yk, SUB(f, t, st->s));
        st->s = t;
        break; }
    case 2: { /* rigorous, Example 3: TWO-SUM(s, y) (Theorem 2), error q to e */
        const double x = ADD(f, st->s, y);
        const double bv = SUB(f, x, st->s), av = SUB(f, x, bv);
        const double q = ADD(f, SUB(f, st->s, av), SUB(f, y, bv));
        st->e = (P->op == 0) ? ADD(f, st->e, q) : ADD(f, st->e, ADD(f, q, ep));
        st->s = x;
        break; }
    }
}

/* working precision of the in-block levels, and of the cross-block levels:
   0 binary64, 1 binary32, 2 binary128 */
static int f_block(const prob_t* P) {
    if (P->dtype == ORC_F64 && P->variant == 3) return 2;
    return P->dtype == ORC_F32 && P->variant != 3;
}
static int f_grid(const prob_t* P)  {
    if (P->dtype == ORC_F64 && P->variant == 3) return 2;
    return P->dtype == ORC_F32 && P->variant == 0;
}
static int twofold(const prob_t* P) { return P->variant == 1 || P->variant == 2 || P->variant >= 4; }

static pr_t tree_fold(int f, int tw, pr_t* ch, int C) {
    for (int w = C / 2; w >= 1; w /= 2)
        for (int c = 0; c < w; ++c) ch[c] = merge(f, tw, ch[c], ch[c + w]);
    return ch[0];
}

/* butterfly over W values (W a power of two <= 32); returns lane 0's pair */
static pr_t butterfly(int f, int tw, pr_t* v, int W) {
    pr_t tmp[32];
    for (int o = W / 2; o >= 1; o /= 2) {
        for (int i = 0; i < W; ++i) tmp[i] = merge(f, tw, v[i], v[i ^ o]);
        memcpy(v, tmp, sizeof(pr_t) * (size_t)W);
    }
    return v[0];
}

/* pairwise tree over k pairs in order: pair j (j a multiple of 2w) takes
   pair j + w for w = 1, 2, 4, ... while j + w < k; the result is pair 0 */
static pr_t pair_tree(int f, int tw, pr_t* p, int64_t k) {
    for (int64_t w = 1; w < k; w *= 2)
        for (int64_t j = 0; j + w < k; j += 2 * w) p[j] = merge(f, tw, p[j], p[j + w]);
    return p[0];
}

static void write_out(const prob_t* P, pr_t r, int out_f64, void* out) {
    if (P->dtype == ORC_F64 && P->variant == 3) {
        double* o = (double*)out;
        o[0] = (double)r.q;
        o[1] = (double)(r.q - (_Float128)o[0]);
        return;
    }
    if (P->dtype == ORC_F64) {
        double* o = (double*)out; o[0] = r.s; o[1] = r.e; return;
    }
    if (out_f64) { double* o = (double*)out; o[0] = r.s; o[1] = r.e; return; }
    float* o = (float*)out;
    if (P->variant == 0) { o[0] = (float)r.s; o[1] = (float)r.e; return; }
    float v = (float)r.s;                         /* RN32(V) */
    double d = (r.s - (double)v) + r.e;           /* binary64: (V - v) + E */
    o[0] = v; o[1] = (float)d;
}

static int is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

/* the pair of a block's B thread pairs: the tree over the threads (binary64
   twofold variants), else the butterfly of each warp and the butterfly over
   the B/32 warp pairs */
static pr_t block_pair(int f, int tw, int tree, pr_t* tp, int block) {
    if (tree) return tree_fold(f, tw, tp, block);
    pr_t wp[32];
    for (int w = 0; w < block / 32; ++w) wp[w] = butterfly(f, tw, &tp[w * 32], 32);
    return butterfly(f, tw, wp, block / 32);
}

int orc_replay_flat(int dtype, int op, int variant, const void* x, const void* y,
                    int64_t n, int block, int unroll, int64_t grid, int out_f64,
                    void* out) {
    if (block < 32 || block > 1024 || !is_pow2(block) || !is_pow2(unroll) || unroll > 16 ||
        grid < 1 || n < 0 || (dtype != ORC_F32 && dtype != ORC_F64) || variant < 0 ||
        variant > 6 ||  op < 0 || op > 1)
        return -1;
    prob_t P = { dtype, op, variant, x, y };
    int V = (dtype == ORC_F32) ? 4 : 2;
    int C = unroll * V;
    int64_t nv = n / V, tail = n - nv * V;
    int64_t Pth = grid * (int64_t)block;
    int fb = f_block(&P), fg = f_grid(&P), tw = twofold(&P);
    const int tree = (dtype == ORC_F64 && tw);       /* binary64 twofold: thread tree */
    pr_t* bp = (pr_t*)malloc(sizeof(pr_t) * (size_t)grid);
    pr_t* tp = (pr_t*)malloc(sizeof(pr_t) * (size_t)block);
    pr_t ch[64];
    if (!bp || !tp) { free(bp); free(tp); return -1; }
    for (int64_t b = 0; b < grid; ++b) {
        for (int t = 0; t < block; ++t) {
            int64_t g = b * block + t;
            for (int c = 0; c < C; ++c) { ch[c].s = 0.0; ch[c].e = 0.0; ch[c].q = 0; }
            for (int64_t m = 0;; ++m) {
                int64_t j = g + Pth * m;
                if (j >= nv) break;
                for (int l = 0; l < V; ++l) feed(&P, &ch[(m % unroll) * V + l], j * V + l);
            }
            if (tail > 0 && g == nv % Pth) {
                int64_t m = nv / Pth;
                for (int l = 0; l < tail; ++l) feed(&P, &ch[(m % unroll) * V + l], nv * V + l);
            }
            tp[t] = tree_fold(fb, tw, ch, C);
        }
        bp[b] = block_pair(fb, tw, tree, tp, block);
    }
    /* grid fold: the block pairs widen exactly to the grid precision */
    pr_t res;
    {
        for (int t = 0; t < block; ++t) {
            pr_t a = { 0.0, 0.0, 0 };
            if (t < grid) {
                a = bp[t];
                for (int64_t i = t + block; i < grid; i += block) a = merge(fg, tw, a, bp[i]);
            }
            tp[t] = a;
        }
        res = block_pair(fg, tw, tree, tp, block);
    }
    write_out(&P, res, out_f64, out);
    free(bp); free(tp);
    return 0;
}

/* ------------------------------------------------------------------ CSR */

static pr_t piece_pair(const prob_t* P, int64_t a, int64_t b, int64_t tile0, int unroll) {
    int V = (P->dtype == ORC_F32) ? 4 : 2;
    int C = unroll * V;
    int fb = f_block(P), tw = twofold(P);
    pr_t lanes[32];
    pr_t* ch = (pr_t*)calloc((size_t)(32 * C), sizeof(pr_t));   /* all (+0, +0) */
    for (int64_t i = a; i < b; ++i) {
        int64_t r = i - tile0, q = r / V;
        int64_t l = q % 32, m = q / 32;
        feed(P, &ch[l * C + (m % unroll) * V + (int)(r % V)], i);
    }
    for (int l = 0; l < 32; ++l) lanes[l] = tree_fold(fb, tw, &ch[l * C], C);
    free(ch);
    return butterfly(fb, tw, lanes, 32);
}

typedef struct {
    prob_t P; const int64_t* off; int64_t nseg; int unroll; int64_t tile; int out_f64;
    void* out; int64_t* next;
} cjob_t;

static void replay_segment(const cjob_t* J, int64_t s) {
    const prob_t* P = &J->P;
    int64_t a = J->off[s], b = J->off[s + 1];
    size_t osz = (P->dtype == ORC_F64 || J->out_f64) ? 16 : 8;
    void* o = (char*)J->out + osz * (size_t)s;
    pr_t res = { 0.0, 0.0, 0 };
    if (b > a) {
        int64_t w0 = a / J->tile, w1 = (b - 1) / J->tile;
        int64_t k = w1 - w0 + 1;
        pr_t* pcs = (pr_t*)malloc(sizeof(pr_t) * (size_t)k);
        for (int64_t w = w0; w <= w1; ++w) {
            int64_t lo = a > w * J->tile ? a : w * J->tile;
            int64_t hi = b < (w + 1) * J->tile ? b : (w + 1) * J->tile;
            pcs[w - w0] = piece_pair(P, lo, hi, w * J->tile, J->unroll);
        }
        if (k == 1) {
            res = pcs[0];
        } else if (k <= 32) {
            pr_t lanes[32];
            for (int l = 0; l < 32; ++l) {
                pr_t z = { 0.0, 0.0, 0 };
                lanes[l] = l < k ? pcs[l] : z;
            }
            res = butterfly(f_grid(P), twofold(P), lanes, 32);
        } else {
            res = pair_tree(f_grid(P), twofold(P), pcs, k);
        }
        free(pcs);
    }
    write_out(P, res, J->out_f64, o);
}

static void* replay_csr_thread(void* p) {
    cjob_t* J = (cjob_t*)p;
    for (;;) {
        int64_t s = __atomic_fetch_add(J->next, 1, __ATOMIC_RELAXED);
        if (s >= J->nseg) break;
        replay_segment(J, s);
    }
    return NULL;
}

int orc_replay_csr(int dtype, int op, int variant, const void* x, const void* y,
                   const int64_t* off, int64_t nseg, int unroll, int64_t tile,
                   int out_f64, int nthreads, void* out) {
    int V = (dtype == ORC_F32) ? 4 : 2;
    if (!is_pow2(unroll) || unroll > 16 || tile < 32 * V || tile % (32 * V) ||
        nseg < 0 || !off || (dtype != ORC_F32 && dtype != ORC_F64) || variant < 0 ||
        variant > 6 ||  op < 0 || op > 1)
        return -1;
    for (int64_t s = 0; s < nseg; ++s) if (off[s] < 0 || off[s + 1] < off[s]) return -1;
    int64_t next = 0;
    cjob_t J = { { dtype, op, variant, x, y }, off, nseg, unroll, tile, out_f64, out, &next };
    if (nthreads <= 0) nthreads = orc_default_threads();
    if (nthreads > 256) nthreads = 256;
    pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
    if (!th) return -1;
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, replay_csr_thread, &J);
    replay_csr_thread(&J);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th);
    return 0;
}

/* ----------------------------------------------------------- rank merge */
/* Merge G shard pairs in rank order: the last step of one vector cut into G
   contiguous shards, each reduced on its own (one GPU or one call each).
   pairs holds G binary64 pairs (V, E): each shard's cross-block pair, for
   binary32 data its binary64 output form.  Twofold variants (fast, rigorous,
   kahan, the literal dots): from pair 0, pair <- merge(pair, pair g) for
   g = 1 .. G-1 with the TWO-SUM merge above, in binary64.  Plain: V + V_g
   in the data type.  Wide: binary32 data V + V_g in binary64; binary64 data
   S <- (S + V_g) + E_g in binary128 from S = +0, output (RN64(S),
   RN64(S - RN64(S))).  G = 0 gives (+0, +0).  Output as write_out above. */
int orc_merge_pairs(int dtype, int variant, const double* pairs, int64_t G, int out_f64,
                    void* out) {
    if ((dtype != ORC_F32 && dtype != ORC_F64) || variant < 0 || variant > 6 || G < 0 ||
        (G > 0 && !pairs) || !out)
        return -1;
    prob_t P = { dtype, 0, variant, NULL, NULL };
    pr_t r = { 0.0, 0.0, 0 };
    if (dtype == ORC_F64 && variant == 3) {
        _Float128 S = 0;
        for (int64_t g = 0; g < G; ++g)
            S = (S + (_Float128)pairs[2 * g]) + (_Float128)pairs[2 * g + 1];
        r.q = S;
    } else if (G > 0) {
        const int f = f_grid(&P), tw = twofold(&P);
        r.s = pairs[0];
        r.e = pairs[1];
        for (int64_t g = 1; g < G; ++g) {
            pr_t b = { pairs[2 * g], pairs[2 * g + 1], 0 };
            r = merge(f, tw, r, b);
        }
    }
    write_out(&P, r, out_f64, out);
    return 0;
}
