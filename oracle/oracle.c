/*
 * oracle.c -- plain, slow CPU oracle for the DET-LSH hot path
 * (DET-LSH / PDET-LSH, arXiv 2603.24920).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * CPU legs of bench.py.  It shares no code with the CUDA path.
 *
 * Written for a reader checking it against the paper: no blocking, fusion or
 * reordering beyond what the paper's definitions state.  Compile with
 * -ffp-contract=off so that every FP32 expression rounds after each operation.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ======================================================================
 * Philox4x32-10.  Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11: ten rounds of the Philox S-box with the two
 * published multipliers, the key bumped by the two Weyl constants between
 * rounds.
 * ====================================================================== */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Stream ids of the Philox counter (third word). */
#define ORC_STREAM_PROJ 2u
#define ORC_STREAM_SAMPLE 3u

/* ======================================================================
 * Eq. 1 (Sec. II-B): each entry of a is drawn from N(0,1).  Row t = i*K + j
 * is h_{ij}.  Pair (2u, 2u+1) of row t comes from one Philox block with
 * counter (u, t, stream 2, 0) and key (seed lo, seed hi) through Box-Muller
 * in FP64, then rounds to FP32.
 * ====================================================================== */
void orc_projection_matrix(int LK, int64_t d, uint64_t seed, float *A) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int t = 0; t < LK; t++) {
        for (int64_t u = 0; 2 * u < d; u++) {
            uint32_t ctr[4] = {(uint32_t)u, (uint32_t)t, ORC_STREAM_PROJ, 0u};
            uint32_t r[4];
            orc_philox4x32_10(ctr, key, r);
            double u1 = ((double)r[0] + 1.0) * 0x1p-32; /* (0, 1] */
            double u2 = (double)r[1] * 0x1p-32;         /* [0, 1) */
            double radius = sqrt(-2.0 * log(u1));
            double theta = 6.283185307179586 * u2;
            float z0 = (float)(radius * cos(theta));
            float z1 = (float)(radius * sin(theta));
            if (z0 == 0.0f) z0 = 0.0f; /* +0 */
            if (z1 == 0.0f) z1 = 0.0f;
            A[(int64_t)t * d + 2 * u] = z0;
            if (2 * u + 1 < d) A[(int64_t)t * d + 2 * u + 1] = z1;
        }
    }
}

/* ======================================================================
 * Eq. 1: h(o) = a . o.  The FP32 value is defined as the exact real dot
 * product rounded once to the nearest FP32 (ties to even).  Computed here
 * with an exact fixed-point big integer: every FP32 value is m * 2^e with an
 * integer m < 2^24 and e >= -149, so every product is an integer times
 * 2^-298 and fits a 640-bit two's-complement accumulator.
 * ====================================================================== */
#define ORC_NCHUNK 20 /* 20 x 32-bit chunks, bit 0 weighs 2^-298 */
#define ORC_BIAS 298

static void orc_fdecompose(float f, int *neg, uint32_t *mant, int *e2) {
    uint32_t b;
    memcpy(&b, &f, 4);
    *neg = (int)(b >> 31);
    uint32_t E = (b >> 23) & 0xffu, F = b & 0x7fffffu;
    if (E == 0) { *mant = F; *e2 = -149; }
    else { *mant = F | 0x800000u; *e2 = (int)E - 150; }
}

static int orc_acc_bit(const int64_t *acc, int pos) {
    return (int)((acc[pos >> 5] >> (pos & 31)) & 1);
}

static void orc_acc_normalise(int64_t *acc) {
    for (int i = 0; i < ORC_NCHUNK - 1; i++) {
        int64_t carry = acc[i] >> 32; /* arithmetic shift: floor division */
        acc[i] = (int64_t)((uint64_t)acc[i] & 0xffffffffu);
        acc[i + 1] += carry;
    }
}

/* Round the exact value acc * 2^-298 to FP32, nearest, ties to even. */
static float orc_acc_round(int64_t *acc) {
    orc_acc_normalise(acc);
    int neg = acc[ORC_NCHUNK - 1] < 0;
    if (neg) {
        for (int i = 0; i < ORC_NCHUNK; i++) acc[i] = -acc[i];
        orc_acc_normalise(acc);
    }
    int top = -1;
    for (int i = ORC_NCHUNK - 1; i >= 0 && top < 0; i--) {
        if (acc[i] != 0) {
            int b = 31;
            while (!((acc[i] >> b) & 1)) b--;
            top = 32 * i + b;
        }
    }
    if (top < 0) return 0.0f;
    int lsb = top - 23;               /* weight of the last kept bit */
    if (lsb < 149) lsb = 149;         /* 2^-149: FP32 subnormal spacing */
    uint32_t mant = 0;
    for (int pos = top; pos >= lsb; pos--) mant = (mant << 1) | (uint32_t)orc_acc_bit(acc, pos);
    int round_bit = (lsb - 1 >= 0) ? orc_acc_bit(acc, lsb - 1) : 0;
    int sticky = 0;
    for (int pos = lsb - 2; pos >= 0 && !sticky; pos--) sticky = orc_acc_bit(acc, pos);
    if (round_bit && (sticky || (mant & 1u))) mant++;
    if (mant == (1u << 24)) { mant >>= 1; lsb++; }
    if (mant == 0) return 0.0f;
    float v = ldexpf((float)mant, lsb - ORC_BIAS);
    return neg ? -v : v;
}

/* acc += a*b (or -= when negate), exactly; a and b finite. */
static void orc_acc_add_product(int64_t *acc, float a, float b, int negate) {
    int na, nx, ea, ex;
    uint32_t ma, mx;
    orc_fdecompose(a, &na, &ma, &ea);
    orc_fdecompose(b, &nx, &mx, &ex);
    if (ma == 0 || mx == 0) return;
    uint64_t m = (uint64_t)ma * (uint64_t)mx; /* < 2^48, exact */
    int off = ea + ex + ORC_BIAS;              /* >= 0 */
    unsigned __int128 v = (unsigned __int128)m << (off & 31);
    int c = off >> 5;
    int64_t p0 = (int64_t)((uint64_t)v & 0xffffffffu);
    int64_t p1 = (int64_t)((uint64_t)(v >> 32) & 0xffffffffu);
    int64_t p2 = (int64_t)(uint64_t)(v >> 64);
    if ((na ^ nx) ^ (negate != 0)) { acc[c] -= p0; acc[c + 1] -= p1; acc[c + 2] -= p2; }
    else                           { acc[c] += p0; acc[c + 1] += p1; acc[c + 2] += p2; }
}

float orc_dot_rn32(const float *a, const float *x, int64_t d) {
    int64_t acc[ORC_NCHUNK];
    memset(acc, 0, sizeof acc);
    for (int64_t i = 0; i < d; i++) orc_acc_add_product(acc, a[i], x[i], 0);
    return orc_acc_round(acc);
}

/* Is ||q - x|| <= R, decided exactly (no rounding anywhere)?  The squared
 * distance expands into products of two floats,
 *     ||q - x||^2 = sum_j (q_j q_j + x_j x_j - q_j x_j - q_j x_j),
 * and the double R is cut exactly into floats R = f_1 + ... + f_m, so R^2 is
 * the sum of the products f_a f_b; both sums go into the exact fixed-point
 * accumulator and the sign of the difference decides.  Returns 1 (within),
 * 0 (beyond), or -1 when R is negative, NaN or too small to be cut into at
 * most six floats.  A radius of 2^127 or more (beyond FP32, +inf included)
 * counts every point as within: the reading shared with the CUDA path. */
int orc_dist2_le(const float *q, const float *x, int64_t d, double R) {
    if (R >= 0x1p127) return 1; /* beyond FP32: every point counts as within */
    if (!(R >= 0.0)) return -1;
    float f[6];
    int m = 0;
    double rest = R;
    while (rest != 0.0 && m < 6) {
        f[m] = (float)rest;
        rest -= (double)f[m]; /* exact: f[m] is rest rounded to 24 bits */
        m++;
    }
    if (rest != 0.0) return -1;
    int64_t acc[ORC_NCHUNK];
    memset(acc, 0, sizeof acc);
    for (int64_t j = 0; j < d; j++) {
        orc_acc_add_product(acc, q[j], q[j], 0);
        orc_acc_add_product(acc, x[j], x[j], 0);
        orc_acc_add_product(acc, q[j], x[j], 1);
        orc_acc_add_product(acc, q[j], x[j], 1);
    }
    for (int a = 0; a < m; a++)
        for (int b = 0; b < m; b++) orc_acc_add_product(acc, f[a], f[b], 1);
    /* acc = ||q - x||^2 - R^2: within when it is negative or zero */
    orc_acc_normalise(acc);
    if (acc[ORC_NCHUNK - 1] < 0) return 1;
    for (int i = 0; i < ORC_NCHUNK; i++)
        if (acc[i] != 0) return 0;
    return 1;
}

void orc_project(const float *X, int64_t n, int64_t d, const float *A, int LK, float *P) {
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < n; p++)
        for (int t = 0; t < LK; t++)
            P[p * LK + t] = orc_dot_rn32(A + (int64_t)t * d, X + p * d, d);
}

/* ======================================================================
 * Sec. III-A: breakpoints come from n_s = 0.1 n randomly sampled points.
 * The paper does not say how it samples.  Reading: point p is sampled iff
 * the first word of Philox(counter (p lo, p hi, stream 3, 0), key seed) is
 * below floor(frac * 2^32).  If fewer than 2*N_r points are drawn, every
 * point is used.
 * ====================================================================== */
int64_t orc_sample(int64_t n, uint64_t seed, double frac, int N_r, int64_t *ids) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    double scaled = floor(frac * 4294967296.0);
    int all = (scaled >= 4294967296.0);
    uint32_t thr = all ? 0u : (uint32_t)scaled;
    int64_t m = 0;
    for (int64_t p = 0; p < n; p++) {
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)((uint64_t)p >> 32), ORC_STREAM_SAMPLE, 0u};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        if (all || r[0] < thr) ids[m++] = p;
    }
    if (m < 2 * (int64_t)N_r) {
        for (int64_t p = 0; p < n; p++) ids[p] = p;
        m = n;
    }
    return m;
}

static int orc_cmp_float(const void *a, const void *b) {
    float x = *(const float *)a, y = *(const float *)b;
    return (x > y) - (x < y);
}

/* ======================================================================
 * Sec. III-A, dynamic encoding scheme: with C_ij sorted ascending (1-based),
 * B(z) = C(floor(n/N_r) * (z-1)) for z = 2..N_r, B(1) = C(1), B(N_r+1) = C(n).
 * Reading: the interior breakpoints use the sorted sample (n -> m, the
 * sample size); with 0-based B[b] = B(b+1) this is B[b] = S[q*b - 1],
 * q = floor(m/N_r) (at least 1, index clamped to m-1).  The two end
 * breakpoints are the minimum and maximum over all n points, so every point
 * lies inside the outer box.  Sorting gives the same order statistics as
 * the paper's QuickSelect rounds.
 * ====================================================================== */
void orc_breakpoints(const float *P, int64_t n, int LK, const int64_t *sample, int64_t m,
                     int N_r, float *B) {
    float *v = (float *)malloc(sizeof(float) * (size_t)(m > 0 ? m : 1));
    for (int t = 0; t < LK; t++) {
        for (int64_t i = 0; i < m; i++) v[i] = P[sample[i] * LK + t];
        qsort(v, (size_t)m, sizeof(float), orc_cmp_float);
        int64_t q = m / N_r;
        if (q < 1) q = 1;
        float *Bt = B + (int64_t)t * (N_r + 1);
        for (int b = 1; b < N_r; b++) {
            int64_t idx = q * b - 1;
            if (idx > m - 1) idx = m - 1;
            Bt[b] = v[idx];
        }
        float mn = P[t], mx = P[t];
        for (int64_t p = 1; p < n; p++) {
            float h = P[p * LK + t];
            if (h < mn) mn = h;
            if (h > mx) mx = h;
        }
        Bt[0] = mn;
        Bt[N_r] = mx;
    }
    free(v);
}

/* Static encoding scheme (Sec. III-A): breakpoints b_1..b_{N_r-1} cut the
 * N(0,1) density into N_r intervals of equal mass 1/N_r, b_0 = -inf and
 * b_{N_r} = +inf, the same for every projected dimension.  The quantile is
 * found by bisection on Phi(x) = erfc(-x/sqrt 2)/2 down to adjacent doubles
 * in the left half (the right half by symmetry), keeping the one whose Phi is
 * nearer to z/N_r, then rounded to FP32. */
static double orc_norm_quantile(double p) {
    /* symmetric: Phi^-1(1 - p) = -Phi^-1(p), Phi^-1(1/2) = 0 exactly (near 0
     * the rounded Phi is flat over a relatively wide interval) */
    if (p == 0.5) return 0.0;
    if (p > 0.5) return -orc_norm_quantile(1.0 - p);
    double lo = -40.0, hi = 0.0;
    for (int it = 0; it < 2000; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (0.5 * erfc(-mid / sqrt(2.0)) < p) lo = mid; else hi = mid;
    }
    double elo = fabs(0.5 * erfc(-lo / sqrt(2.0)) - p);
    double ehi = fabs(0.5 * erfc(-hi / sqrt(2.0)) - p);
    return elo < ehi ? lo : hi;
}

void orc_static_breakpoints(int LK, int N_r, float *B) {
    for (int t = 0; t < LK; t++) {
        float *Bt = B + (int64_t)t * (N_r + 1);
        for (int z = 1; z < N_r; z++) Bt[z] = (float)orc_norm_quantile((double)z / (double)N_r);
        Bt[0] = -INFINITY;
        Bt[N_r] = INFINITY;
    }
}

/* ======================================================================
 * Alg. 1: find b with B(b) <= h <= B(b+1) and store the b-th symbol.  The
 * closed interval admits two b at a breakpoint; reading: the first such b,
 * so the 0-based code is the number of interior breakpoints strictly below h.
 * Counted by a linear scan (BinarySearch returns the same index).
 * ====================================================================== */
void orc_encode(const float *P, int64_t n, int LK, const float *B, int N_r, uint8_t *codes) {
    for (int64_t p = 0; p < n; p++) {
        for (int t = 0; t < LK; t++) {
            const float *Bt = B + (int64_t)t * (N_r + 1);
            float h = P[p * LK + t];
            int code = 0;
            for (int b = 1; b < N_r; b++)
                if (Bt[b] < h) code++;
            codes[p * LK + t] = (uint8_t)code;
        }
    }
}

/* ======================================================================
 * Lemma 2 / Lemma 3 / Eq. 2 (Sec. V-A): eps^2 = chi^2_{alpha1}(K), the upper
 * alpha1-quantile of chi^2(K), with L = -1/ln(alpha1), i.e.
 * alpha1 = exp(-1/L).  Upper tail of chi^2(K):
 *   K even: exp(-x/2) * sum_{i<K/2} (x/2)^i / i!
 *   K odd : erfc(sqrt(x/2)) + exp(-x/2) * sqrt(2x/pi) *
 *           sum_{i=1}^{(K-1)/2} x^(i-1) / (1*3*...*(2i-1))
 * Solved by bisection in FP64.
 * ====================================================================== */
double orc_chi2_sf(double x, int K) {
    if (x <= 0.0) return 1.0;
    if (K % 2 == 0) {
        double term = 1.0, sum = 1.0;
        for (int i = 1; i < K / 2; i++) {
            term *= (x / 2.0) / (double)i;
            sum += term;
        }
        return exp(-x / 2.0) * sum;
    }
    double sum = 0.0, term = 1.0;
    for (int i = 1; i <= (K - 1) / 2; i++) {
        if (i > 1) term *= x / (double)(2 * i - 1);
        sum += term;
    }
    return erfc(sqrt(x / 2.0)) + exp(-x / 2.0) * sqrt(2.0 * x / 3.141592653589793) * sum;
}

double orc_eps2(int K, int L) {
    double alpha1 = exp(-1.0 / (double)L);
    double lo = 0.0, hi = 1.0;
    while (orc_chi2_sf(hi, K) > alpha1) hi *= 2.0;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_chi2_sf(mid, K) > alpha1) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Radius grid for the magic r_min (Sec. V-B1).  Reading: r_j = r0 * c^j with
 * r0 = 1, j = -127..127; a leaf is inside the range query of radius r_j iff
 * its squared lower bound is <= T(j) = fp32(eps^2 r_j^2); T(127) = +inf so
 * the largest radius takes every leaf. */
void orc_level_table(double eps2, double c, float *T) {
    for (int i = 0; i < ORC_NLEV; i++) {
        int j = i + ORC_JMIN;
        T[i] = (float)(eps2 * pow(c, 2.0 * (double)j));
    }
    T[ORC_NLEV - 1] = INFINITY;
}

/* ======================================================================
 * DE-Tree (Alg. 2, Sec. III-B).  Pointer-based: the root has 2^K first-layer
 * children (one bit per dimension), every deeper node splits one dimension
 * by its next code bit.
 * ====================================================================== */
typedef struct onode {
    int64_t *ids;           /* members (leaves; internal nodes drop theirs) */
    int64_t cnt, cap;
    uint8_t nb[16];         /* prefix length in bits, per dimension */
    uint8_t prefix[16];     /* prefix value, per dimension */
    uint8_t lo[16], hi[16]; /* box, in regions, per dimension */
    struct onode *child[2];
    int split_dim;          /* -1 for a leaf */
    int64_t leaf_id;
} onode;

typedef struct {
    onode **first; /* 2^K first-layer nodes, NULL when empty */
    int64_t nleaves;
    onode **leaves; /* canonical order */
} otree;

struct orc_index {
    int64_t n, d;
    int L, K, N_r, bbits, M, box_mode;
    uint64_t seed;
    double frac;
    float *X, *A, *P, *B;
    uint8_t *codes;
    int64_t *sample, m;
    otree *trees;
    double eps2;
};

static const uint8_t *orc_code_row(const orc_index *ix, int t, int64_t p) {
    return ix->codes + p * (int64_t)(ix->L * ix->K) + (int64_t)t * ix->K;
}

static void orc_node_push(onode *nd, int64_t p) {
    if (nd->cnt == nd->cap) {
        nd->cap = nd->cap ? 2 * nd->cap : 8;
        nd->ids = (int64_t *)realloc(nd->ids, sizeof(int64_t) * (size_t)nd->cap);
    }
    nd->ids[nd->cnt++] = p;
}

/* Next code bit of dimension j for a node whose prefix has nb bits. */
static int orc_next_bit(const orc_index *ix, uint8_t code, int nb) {
    return (code >> (ix->bbits - 1 - nb)) & 1;
}

/* Node box (Sec. IV-C): the regions covered by the node's iSAX prefix; in
 * tight mode the min/max codes of its members. */
static void orc_node_box(const orc_index *ix, int t, onode *nd) {
    for (int j = 0; j < ix->K; j++) {
        int free_bits = ix->bbits - nd->nb[j];
        nd->lo[j] = (uint8_t)(nd->prefix[j] << free_bits);
        nd->hi[j] = (uint8_t)((nd->prefix[j] << free_bits) + (1 << free_bits) - 1);
    }
    if (ix->box_mode == 1 && nd->cnt > 0) {
        for (int j = 0; j < ix->K; j++) { nd->lo[j] = 255; nd->hi[j] = 0; }
        for (int64_t i = 0; i < nd->cnt; i++) {
            const uint8_t *c = orc_code_row(ix, t, nd->ids[i]);
            for (int j = 0; j < ix->K; j++) {
                if (c[j] < nd->lo[j]) nd->lo[j] = c[j];
                if (c[j] > nd->hi[j]) nd->hi[j] = c[j];
            }
        }
    }
}

/* Split rule (Sec. III-B): the dimension that most evenly partitions the
 * node's points, i.e. argmin |n0 - n1| over dimensions with bits left;
 * reading: ties go to the smallest dimension.  Returns -1 if none. */
static int orc_choose_split(const orc_index *ix, int t, const onode *nd) {
    int best = -1;
    int64_t best_diff = 0;
    for (int j = 0; j < ix->K; j++) {
        if (nd->nb[j] >= ix->bbits) continue;
        int64_t n1 = 0;
        for (int64_t i = 0; i < nd->cnt; i++)
            n1 += orc_next_bit(ix, orc_code_row(ix, t, nd->ids[i])[j], nd->nb[j]);
        int64_t diff = llabs(nd->cnt - 2 * n1);
        if (best < 0 || diff < best_diff) { best = j; best_diff = diff; }
    }
    return best;
}

static onode *orc_new_child(const onode *parent, int j, int bit) {
    onode *c = (onode *)calloc(1, sizeof(onode));
    memcpy(c->nb, parent->nb, 16);
    memcpy(c->prefix, parent->prefix, 16);
    c->nb[j] = (uint8_t)(parent->nb[j] + 1);
    c->prefix[j] = (uint8_t)((parent->prefix[j] << 1) | bit);
    c->split_dim = -1;
    return c;
}

/* Split a node into two children on dimension j; members keep their order. */
static void orc_split(const orc_index *ix, int t, onode *nd, int j, int keep_empty) {
    onode *c0 = orc_new_child(nd, j, 0), *c1 = orc_new_child(nd, j, 1);
    for (int64_t i = 0; i < nd->cnt; i++) {
        int64_t p = nd->ids[i];
        if (orc_next_bit(ix, orc_code_row(ix, t, p)[j], nd->nb[j])) orc_node_push(c1, p);
        else orc_node_push(c0, p);
    }
    free(nd->ids);
    nd->ids = NULL;
    nd->cnt = nd->cap = 0; /* members now live in the children */
    nd->split_dim = j;
    if (!keep_empty && c0->cnt == 0) { free(c0); c0 = NULL; }
    if (!keep_empty && c1->cnt == 0) { free(c1); c1 = NULL; }
    nd->child[0] = c0;
    nd->child[1] = c1;
}

/* Canonical bulk build.  Reading of Alg. 2 (which depends on insertion order
 * and leaves max_size open): a node is split iff it holds more than M points
 * and some dimension has bits left; empty children are dropped. */
static void orc_build_bulk(const orc_index *ix, int t, onode *nd) {
    orc_node_box(ix, t, nd);
    if (nd->cnt <= ix->M) return;
    int j = orc_choose_split(ix, t, nd);
    if (j < 0) return;
    orc_split(ix, t, nd, j, 0);
    for (int b = 0; b < 2; b++)
        if (nd->child[b]) orc_build_bulk(ix, t, nd->child[b]);
}

/* Literal Alg. 2: insert <ep, pos> in order; while the target leaf holds
 * max_size points, split it and descend to the new target leaf. */
static void orc_insert(const orc_index *ix, int t, onode *leaf, int64_t p) {
    const uint8_t *c = orc_code_row(ix, t, p);
    onode *nd = leaf;
    for (;;) {
        while (nd->split_dim >= 0) {
            int j = nd->split_dim;
            nd = nd->child[orc_next_bit(ix, c[j], nd->nb[j])];
        }
        if (nd->cnt < ix->M) break;
        int j = orc_choose_split(ix, t, nd);
        if (j < 0) break; /* nothing left to split on: the leaf grows */
        orc_split(ix, t, nd, j, 1);
    }
    orc_node_push(nd, p);
}

/* Boxes of an insertion-built tree, bottom-up.  Returns 1 if the subtree
 * holds a point.  Tight mode: an internal box is the hull of its non-empty
 * children. */
static int orc_boxes_rec(const orc_index *ix, int t, onode *nd) {
    if (nd->split_dim < 0) {
        orc_node_box(ix, t, nd);
        return nd->cnt > 0;
    }
    int nonempty[2] = {0, 0};
    for (int b = 0; b < 2; b++)
        if (nd->child[b]) nonempty[b] = orc_boxes_rec(ix, t, nd->child[b]);
    orc_node_box(ix, t, nd); /* prefix box */
    if (ix->box_mode == 1) {
        int first = 1;
        for (int b = 0; b < 2; b++) {
            if (!nonempty[b]) continue;
            const onode *ch = nd->child[b];
            for (int j = 0; j < ix->K; j++) {
                if (first || ch->lo[j] < nd->lo[j]) nd->lo[j] = ch->lo[j];
                if (first || ch->hi[j] > nd->hi[j]) nd->hi[j] = ch->hi[j];
            }
            first = 0;
        }
    }
    return nonempty[0] || nonempty[1];
}

static void orc_collect_leaves(otree *T, onode *nd) {
    if (nd->split_dim < 0) {
        if (nd->cnt > 0) {
            nd->leaf_id = T->nleaves;
            T->leaves[T->nleaves++] = nd;
        } else {
            nd->leaf_id = -1;
        }
        return;
    }
    for (int b = 0; b < 2; b++)
        if (nd->child[b]) orc_collect_leaves(T, nd->child[b]);
}

static void orc_free_node(onode *nd) {
    if (!nd) return;
    orc_free_node(nd->child[0]);
    orc_free_node(nd->child[1]);
    free(nd->ids);
    free(nd);
}

static int64_t orc_first_key(const orc_index *ix, int t, int64_t p) {
    const uint8_t *c = orc_code_row(ix, t, p);
    int64_t key = 0;
    for (int j = 0; j < ix->K; j++)
        key |= (int64_t)((c[j] >> (ix->bbits - 1)) & 1) << (ix->K - 1 - j);
    return key;
}

static void orc_build_tree(orc_index *ix, int t, int insertion_order) {
    otree *T = &ix->trees[t];
    int64_t nfirst = (int64_t)1 << ix->K;
    T->first = (onode **)calloc((size_t)nfirst, sizeof(onode *));
    /* Alg. 2: 2^K first-layer nodes, each dimension split into 0* and 1*. */
    for (int64_t p = 0; p < ix->n; p++) {
        int64_t key = orc_first_key(ix, t, p);
        onode *nd = T->first[key];
        if (!nd) {
            nd = (onode *)calloc(1, sizeof(onode));
            const uint8_t *c = orc_code_row(ix, t, p);
            for (int j = 0; j < ix->K; j++) {
                nd->nb[j] = 1;
                nd->prefix[j] = (uint8_t)((c[j] >> (ix->bbits - 1)) & 1);
            }
            nd->split_dim = -1;
            T->first[key] = nd;
        }
        if (insertion_order) orc_insert(ix, t, nd, p);
        else orc_node_push(nd, p);
    }
    for (int64_t key = 0; key < nfirst; key++) {
        onode *nd = T->first[key];
        if (!nd) continue;
        if (insertion_order) orc_boxes_rec(ix, t, nd);
        else orc_build_bulk(ix, t, nd);
    }
    T->leaves = (onode **)malloc(sizeof(onode *) * (size_t)(ix->n > 0 ? ix->n : 1));
    T->nleaves = 0;
    for (int64_t key = 0; key < nfirst; key++)
        if (T->first[key]) orc_collect_leaves(T, T->first[key]);
}

orc_index *orc_index_build(const float *X, int64_t n, int64_t d, int L, int K, int N_r,
                           uint64_t seed, double frac, int M, int box_mode,
                           int insertion_order, int encoding) {
    orc_index *ix = (orc_index *)calloc(1, sizeof(orc_index));
    ix->n = n; ix->d = d; ix->L = L; ix->K = K; ix->N_r = N_r; ix->seed = seed;
    ix->frac = frac; ix->M = M; ix->box_mode = box_mode;
    ix->bbits = 0;
    while ((1 << ix->bbits) < N_r) ix->bbits++;
    int LK = L * K;
    ix->X = (float *)malloc(sizeof(float) * (size_t)(n * d));
    memcpy(ix->X, X, sizeof(float) * (size_t)(n * d));
    ix->A = (float *)malloc(sizeof(float) * (size_t)(LK * d));
    orc_projection_matrix(LK, d, seed, ix->A);
    ix->P = (float *)malloc(sizeof(float) * (size_t)(n * LK));
    orc_project(ix->X, n, d, ix->A, LK, ix->P);
    ix->sample = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    ix->B = (float *)malloc(sizeof(float) * (size_t)(LK * (N_r + 1)));
    if (encoding == 1) {  /* static scheme: no sample */
        ix->m = 0;
        orc_static_breakpoints(LK, N_r, ix->B);
    } else {              /* dynamic scheme */
        ix->m = orc_sample(n, seed, frac, N_r, ix->sample);
        orc_breakpoints(ix->P, n, LK, ix->sample, ix->m, N_r, ix->B);
    }
    ix->codes = (uint8_t *)malloc((size_t)(n * LK));
    orc_encode(ix->P, n, LK, ix->B, N_r, ix->codes);
    ix->trees = (otree *)calloc((size_t)L, sizeof(otree));
    for (int t = 0; t < L; t++) orc_build_tree(ix, t, insertion_order);
    ix->eps2 = orc_eps2(K, L);
    return ix;
}

void orc_index_free(orc_index *ix) {
    if (!ix) return;
    for (int t = 0; t < ix->L; t++) {
        otree *T = &ix->trees[t];
        if (T->first) {
            for (int64_t key = 0; key < ((int64_t)1 << ix->K); key++) orc_free_node(T->first[key]);
            free(T->first);
        }
        free(T->leaves);
    }
    free(ix->trees);
    free(ix->X); free(ix->A); free(ix->P); free(ix->B); free(ix->codes); free(ix->sample);
    free(ix);
}

int64_t orc_index_sample_size(const orc_index *ix) { return ix->m; }
int64_t orc_index_num_leaves(const orc_index *ix, int t) { return ix->trees[t].nleaves; }

void orc_index_export_arrays(const orc_index *ix, float *A, float *B, uint8_t *codes,
                             float *P, int64_t *sample) {
    int LK = ix->L * ix->K;
    if (A) memcpy(A, ix->A, sizeof(float) * (size_t)(LK * ix->d));
    if (B) memcpy(B, ix->B, sizeof(float) * (size_t)(LK * (ix->N_r + 1)));
    if (codes) memcpy(codes, ix->codes, (size_t)(ix->n * LK));
    if (P) memcpy(P, ix->P, sizeof(float) * (size_t)(ix->n * LK));
    if (sample) memcpy(sample, ix->sample, sizeof(int64_t) * (size_t)ix->m);
}

void orc_index_export_tree(const orc_index *ix, int t, int64_t *perm, int64_t *leaf_begin,
                           uint8_t *box_lo, uint8_t *box_hi, uint8_t *nbits,
                           int64_t *leaf_of) {
    const otree *T = &ix->trees[t];
    int64_t pos = 0;
    for (int64_t l = 0; l < T->nleaves; l++) {
        const onode *nd = T->leaves[l];
        if (leaf_begin) leaf_begin[l] = pos;
        for (int64_t i = 0; i < nd->cnt; i++) {
            if (perm) perm[pos] = nd->ids[i];
            if (leaf_of) leaf_of[nd->ids[i]] = l;
            pos++;
        }
        for (int j = 0; j < ix->K; j++) {
            if (box_lo) box_lo[l * ix->K + j] = nd->lo[j];
            if (box_hi) box_hi[l * ix->K + j] = nd->hi[j];
            if (nbits) nbits[l * ix->K + j] = nd->nb[j];
        }
    }
    if (leaf_begin) leaf_begin[T->nleaves] = pos;
}

void orc_index_level_table(const orc_index *ix, double c, float *T) {
    orc_level_table(ix->eps2, c, T);
}

/* ======================================================================
 * Query phase.
 * ====================================================================== */

/* Lower bound between q' and a node box (Sec. IV-C): per dimension the gap
 * from q'_j to the box's breakpoint interval [B(lo), B(hi+1)] (zero inside),
 * then the sum of squares.  FP32, dimensions in ascending order. */
static float orc_lb2(const orc_index *ix, int t, const float *qp, const uint8_t *lo,
                     const uint8_t *hi) {
    float acc = 0.0f;
    for (int j = 0; j < ix->K; j++) {
        const float *Bt = ix->B + (int64_t)(t * ix->K + j) * (ix->N_r + 1);
        float g_low = Bt[lo[j]] - qp[j];
        float g_high = qp[j] - Bt[hi[j] + 1];
        float gap = 0.0f;
        if (g_low > gap) gap = g_low;
        if (g_high > gap) gap = g_high;
        acc = acc + gap * gap;
    }
    return acc;
}

typedef struct {
    float lb2;
    int64_t leaf_id;
    const onode *leaf;
} orc_hit;

typedef struct {
    orc_hit *v;
    int64_t n, cap;
} orc_hits;

static void orc_hits_push(orc_hits *h, orc_hit x) {
    if (h->n == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 64;
        h->v = (orc_hit *)realloc(h->v, sizeof(orc_hit) * (size_t)h->cap);
    }
    h->v[h->n++] = x;
}

/* Alg. 3 with optimisation (1) of Sec. VI-B2: traverse the subtree, prune a
 * node whose lower bound exceeds r', take a leaf whole when its lower bound
 * is within r'.  Comparisons are on squared values against T = fp32((eps r)^2). */
static void orc_range_rec(const orc_index *ix, int t, const float *qp, const onode *nd,
                          float T, orc_hits *out) {
    float lb2 = orc_lb2(ix, t, qp, nd->lo, nd->hi);
    if (lb2 > T) return;
    if (nd->split_dim < 0) {
        if (nd->cnt > 0) {
            orc_hit h = {lb2, nd->leaf_id, nd};
            orc_hits_push(out, h);
        }
        return;
    }
    for (int b = 0; b < 2; b++)
        if (nd->child[b]) orc_range_rec(ix, t, qp, nd->child[b], T, out);
}

static void orc_range_query(const orc_index *ix, int t, const float *qp, float T,
                            orc_hits *out) {
    out->n = 0;
    const otree *tr = &ix->trees[t];
    for (int64_t key = 0; key < ((int64_t)1 << ix->K); key++)
        if (tr->first[key]) orc_range_rec(ix, t, qp, tr->first[key], T, out);
}

static int orc_cmp_hit(const void *a, const void *b) {
    const orc_hit *x = (const orc_hit *)a, *y = (const orc_hit *)b;
    if (x->lb2 < y->lb2) return -1;
    if (x->lb2 > y->lb2) return 1;
    return (x->leaf_id > y->leaf_id) - (x->leaf_id < y->leaf_id);
}

typedef struct {
    double dist;
    int64_t id;
} orc_cand;

static int orc_cmp_cand(const void *a, const void *b) {
    const orc_cand *x = (const orc_cand *)a, *y = (const orc_cand *)b;
    if (x->dist < y->dist) return -1;
    if (x->dist > y->dist) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

static double orc_dist(const float *q, const float *x, int64_t d) {
    double s = 0.0;
    for (int64_t i = 0; i < d; i++) {
        double diff = (double)q[i] - (double)x[i];
        s += diff * diff;
    }
    return sqrt(s);
}

/* |S| after the union over all L trees at radius index j (the range queries
 * of Alg. 5 at one radius, without its early return). */
static int64_t orc_union_size(const orc_index *ix, const float *qproj, float T, uint8_t *mark,
                              orc_hits *hits) {
    memset(mark, 0, (size_t)ix->n);
    int64_t cnt = 0;
    for (int t = 0; t < ix->L; t++) {
        orc_range_query(ix, t, qproj + t * ix->K, T, hits);
        for (int64_t h = 0; h < hits->n; h++) {
            const onode *lf = hits->v[h].leaf;
            for (int64_t i = 0; i < lf->cnt; i++)
                if (!mark[lf->ids[i]]) { mark[lf->ids[i]] = 1; cnt++; }
        }
    }
    return cnt;
}

/* ----------------------------------------------------------------------
 * Alg. 3 as printed (before the optimisations of Sec. VI-B2) and Alg. 4.
 * ---------------------------------------------------------------------- */

/* Upper bound between q' and a node box (Sec. IV-C, Fig. 6): per dimension
 * the distance from q'_j to the farther edge of the interval [B(lo), B(hi+1)],
 * then the sum of squares.  FP32, dimensions in ascending order. */
static float orc_ub2(const orc_index *ix, int t, const float *qp, const uint8_t *lo,
                     const uint8_t *hi) {
    float acc = 0.0f;
    for (int j = 0; j < ix->K; j++) {
        const float *Bt = ix->B + (int64_t)(t * ix->K + j) * (ix->N_r + 1);
        float to_low = fabsf(Bt[lo[j]] - qp[j]);
        float to_high = fabsf(Bt[hi[j] + 1] - qp[j]);
        float far = to_low > to_high ? to_low : to_high;
        acc = acc + far * far;
    }
    return acc;
}

/* Both node bounds of one box given directly by its breakpoints (K rows of
 * N_r + 1), so that tests can check them on hand-worked boxes. */
void orc_box_bounds(const float *B, int K, int N_r, const float *qp, const uint8_t *lo,
                    const uint8_t *hi, float *lb2, float *ub2) {
    orc_index one;
    memset(&one, 0, sizeof one);
    one.B = (float *)B;
    one.K = K;
    one.N_r = N_r;
    one.L = 1;
    *lb2 = orc_lb2(&one, 0, qp, lo, hi);
    *ub2 = orc_ub2(&one, 0, qp, lo, hi);
}

/* Squared distance between a point's projection H_t(o) and q'_t in tree t's
 * projected space: FP32, dimensions in ascending order. */
static float orc_proj_dist2(const orc_index *ix, int t, const float *qp, int64_t p) {
    const float *po = ix->P + p * (int64_t)(ix->L * ix->K) + (int64_t)t * ix->K;
    float acc = 0.0f;
    for (int j = 0; j < ix->K; j++) {
        float dj = po[j] - qp[j];
        acc = acc + dj * dj;
    }
    return acc;
}

/* Alg. 3 with the pruning rules of Sec. IV-C: a node whose lower bound
 * exceeds r' is discarded; a leaf whose upper bound is within r' gives all
 * its points; otherwise its points are examined one by one and those within
 * r' of q' (projected distance) are added.  Squared values against R2. */
static void orc_range_exact_rec(const orc_index *ix, int t, const float *qp, const onode *nd,
                                float R2, int64_t *out, int64_t *nout) {
    if (orc_lb2(ix, t, qp, nd->lo, nd->hi) > R2) return;
    if (nd->split_dim < 0) {
        int whole = orc_ub2(ix, t, qp, nd->lo, nd->hi) <= R2;
        for (int64_t i = 0; i < nd->cnt; i++) {
            int64_t p = nd->ids[i];
            if (whole || orc_proj_dist2(ix, t, qp, p) <= R2) out[(*nout)++] = p;
        }
        return;
    }
    for (int b = 0; b < 2; b++)
        if (nd->child[b]) orc_range_exact_rec(ix, t, qp, nd->child[b], R2, out, nout);
}

static void orc_query_proj(const orc_index *ix, const float *q, float *qproj) {
    for (int t = 0; t < ix->L * ix->K; t++)
        qproj[t] = orc_dot_rn32(ix->A + (int64_t)t * ix->d, q, ix->d);
}

int64_t orc_index_range_exact(const orc_index *ix, int t, const float *q, double r,
                              int64_t *out) {
    float qproj[256];
    orc_query_proj(ix, q, qproj);
    const float R2 = (float)(ix->eps2 * r * r); /* (eps r)^2, rounded once */
    const otree *tr = &ix->trees[t];
    int64_t nout = 0;
    for (int64_t key = 0; key < ((int64_t)1 << ix->K); key++)
        if (tr->first[key])
            orc_range_exact_rec(ix, t, qproj + t * ix->K, tr->first[key], R2, out, &nout);
    return nout;
}

void orc_index_leaf_ub2(const orc_index *ix, int t, const float *q, float *ub2) {
    float qproj[256];
    orc_query_proj(ix, q, qproj);
    const otree *T = &ix->trees[t];
    for (int64_t l = 0; l < T->nleaves; l++)
        ub2[l] = orc_ub2(ix, t, qproj + t * ix->K, T->leaves[l]->lo, T->leaves[l]->hi);
}

int orc_index_rc_ann(const orc_index *ix, const float *q, double r, double beta, double c,
                     int optimised, int64_t *id, double *dist, int64_t *S_out,
                     int64_t *S_size, int *tree_stop) {
    const int64_t n = ix->n;
    const int64_t need = (int64_t)ceil(beta * (double)n) + 1; /* beta*n + 1 */
    float qproj[256];
    orc_query_proj(ix, q, qproj);
    const float R2 = (float)(ix->eps2 * r * r);
    uint8_t *mark = (uint8_t *)calloc((size_t)n, 1);
    int64_t *Rt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    int64_t ns = 0;
    int stop = -1;
    for (int t = 0; t < ix->L; t++) {
        const otree *tr = &ix->trees[t];
        int64_t nr = 0;
        if (optimised) {  /* optimisation (1) of Sec. VI-B2: leaves whole by lower bound */
            orc_hits hits = {0};
            orc_range_query(ix, t, qproj + t * ix->K, R2, &hits);
            for (int64_t h = 0; h < hits.n; h++)
                for (int64_t i = 0; i < hits.v[h].leaf->cnt; i++) Rt[nr++] = hits.v[h].leaf->ids[i];
            free(hits.v);
        } else {
            for (int64_t key = 0; key < ((int64_t)1 << ix->K); key++)
                if (tr->first[key])
                    orc_range_exact_rec(ix, t, qproj + t * ix->K, tr->first[key], R2, Rt, &nr);
        }
        for (int64_t i = 0; i < nr; i++)
            if (!mark[Rt[i]]) { mark[Rt[i]] = 1; S[ns++] = Rt[i]; }
        if (ns >= need) { stop = t; break; }
    }
    /* the point of S closest to q (FP64 distances, ties by smaller id) */
    int64_t best = -1;
    double bd = INFINITY;
    for (int64_t i = 0; i < ns; i++) {
        double dd = orc_dist(q, ix->X + S[i] * ix->d, ix->d);
        if (dd < bd || (dd == bd && S[i] < best)) { bd = dd; best = S[i]; }
    }
    if (stop < 0 && !(best >= 0 && bd <= c * r)) { best = -1; bd = INFINITY; }
    *id = best;
    *dist = bd;
    if (S_out) for (int64_t i = 0; i < ns; i++) S_out[i] = S[i];
    if (S_size) *S_size = ns;
    if (tree_stop) *tree_stop = stop;
    free(mark); free(Rt); free(S);
    return 0;
}

int orc_index_query_ex(const orc_index *ix, const float *q, int k, double beta, double c,
                       int per_tree, int64_t *ids, double *dists, int64_t *S_out,
                       int64_t *S_size, int *jstar, int *istar);

int orc_index_query(const orc_index *ix, const float *q, int k, double beta, double c,
                    int64_t *ids, double *dists, int64_t *S_out, int64_t *S_size,
                    int *jstar, int *istar) {
    return orc_index_query_ex(ix, q, k, beta, c, 0, ids, dists, S_out, S_size, jstar, istar);
}

/* per_tree = 1: Alg. 5 without the priority queue of Sec. VI-B2: a tree's
 * range query joins S whole and the budget is checked after each tree
 * (the check as Alg. 5 prints it). */
int orc_index_query_ex(const orc_index *ix, const float *q, int k, double beta, double c,
                       int per_tree, int64_t *ids, double *dists, int64_t *S_out,
                       int64_t *S_size, int *jstar, int *istar) {
    int64_t n = ix->n;
    if (k < 1 || k > n) return -1;
    int LK = ix->L * ix->K;
    int64_t tau = (int64_t)ceil(beta * (double)n) + k; /* beta*n + k */
    orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)n);
    int64_t ns = 0;
    int js = 127, is = -1;
    if (tau > n) {
        /* The candidate budget can never be met: Alg. 5 ends through its
         * second condition once S is the whole dataset, so S = D. */
        for (int64_t p = 0; p < n; p++) { cand[ns].id = p; ns++; }
        if (S_out) for (int64_t p = 0; p < n; p++) S_out[p] = p;
    } else {
        float qproj[256];
        for (int t = 0; t < LK; t++) qproj[t] = orc_dot_rn32(ix->A + (int64_t)t * ix->d, q, ix->d);
        float T[ORC_NLEV];
        orc_level_table(ix->eps2, c, T);
        uint8_t *mark = (uint8_t *)malloc((size_t)n);
        orc_hits hits = {0};
        /* Magic r_min (Sec. V-B1): the smallest grid radius whose union
         * reaches beta*n + k; the union size is monotone in r, so bisect. */
        int lo = -1, hi = ORC_NLEV - 1; /* N(hi) >= tau always (T = inf) */
        while (hi - lo > 1) {
            int mid = (lo + hi) / 2;
            if (orc_union_size(ix, qproj, T[mid], mark, &hits) >= tau) hi = mid;
            else lo = mid;
        }
        js = hi + ORC_JMIN;
        /* Alg. 5 at r = r_min: trees in order; within a tree the leaves of
         * the range query enter S in ascending lower-bound order, ties by
         * leaf id (the priority queue of Sec. VI-B2); stop as soon as
         * |S| >= beta*n + k. */
        memset(mark, 0, (size_t)n);
        for (int t = 0; t < ix->L && ns < tau; t++) {
            orc_range_query(ix, t, qproj + t * ix->K, T[hi], &hits);
            qsort(hits.v, (size_t)hits.n, sizeof(orc_hit), orc_cmp_hit);
            for (int64_t h = 0; h < hits.n && (per_tree || ns < tau); h++) {
                const onode *lf = hits.v[h].leaf;
                for (int64_t i = 0; i < lf->cnt; i++) {
                    int64_t p = lf->ids[i];
                    if (!mark[p]) {
                        mark[p] = 1;
                        if (S_out) S_out[ns] = p;
                        cand[ns++].id = p;
                    }
                }
                if (!per_tree && ns >= tau) is = t;
            }
            if (per_tree && ns >= tau) is = t;
        }
        free(hits.v);
        free(mark);
    }
    /* Verification: exact distances, top-k by (distance, id). */
    for (int64_t i = 0; i < ns; i++)
        cand[i].dist = orc_dist(q, ix->X + cand[i].id * ix->d, ix->d);
    qsort(cand, (size_t)ns, sizeof(orc_cand), orc_cmp_cand);
    for (int i = 0; i < k; i++) {
        ids[i] = cand[i].id;
        dists[i] = cand[i].dist;
    }
    if (S_size) *S_size = ns;
    if (jstar) *jstar = js;
    if (istar) *istar = is;
    free(cand);
    return 0;
}

/* Alg. 5 run literally from a given r_min (no magic r_min): radii
 * r_i = r_min c^i, i = 0, 1, ...; at each radius the trees in order, leaves
 * of the range query entering S whole in ascending (LB^2, leaf id) order with
 * the check |S| >= beta*n + k after each leaf (condition 1); after the L
 * trees, condition 2: at least k points of S within c*r, each distance
 * compared with c*r exactly (orc_dist2_le; c*r is the FP64 value
 * c * (r_min * c^i)).  S accumulates across radii.  jstop = i of the radius
 * that stopped, istop = the tree for condition 1, -1 for condition 2. */
int orc_index_query_fixed(const orc_index *ix, const float *q, int k, double beta, double c,
                          double r_min, int64_t *ids, double *dists, int64_t *S_out,
                          int64_t *S_size, int *jstop, int *istop) {
    int64_t n = ix->n;
    if (k < 1 || k > n || !(r_min > 0.0)) return -1;
    int64_t tau = (int64_t)ceil(beta * (double)n) + k;
    float qproj[256];
    orc_query_proj(ix, q, qproj);
    uint8_t *mark = (uint8_t *)calloc((size_t)n, 1);
    orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)n);
    orc_hits hits = {0};
    int64_t ns = 0;
    int js = -1, is = -1, bad = 0;
    for (int i = 0; i < ORC_NLEV && js < 0; i++) {
        const float Ti = (i == ORC_NLEV - 1) ? INFINITY
                         : (float)(ix->eps2 * r_min * r_min * pow(c, 2.0 * (double)i));
        for (int t = 0; t < ix->L && js < 0; t++) {
            orc_range_query(ix, t, qproj + t * ix->K, Ti, &hits);
            qsort(hits.v, (size_t)hits.n, sizeof(orc_hit), orc_cmp_hit);
            for (int64_t h = 0; h < hits.n && js < 0; h++) {
                const onode *lf = hits.v[h].leaf;
                for (int64_t e = 0; e < lf->cnt; e++) {
                    int64_t p = lf->ids[e];
                    if (!mark[p]) {
                        mark[p] = 1;
                        cand[ns].id = p;
                        cand[ns].dist = orc_dist(q, ix->X + p * ix->d, ix->d);
                        if (S_out) S_out[ns] = p;
                        ns++;
                    }
                }
                if (ns >= tau) { js = i; is = t; }
            }
        }
        if (js < 0) {
            /* condition 2, decided exactly; the last radius is unbounded (its
             * range query already takes every leaf) */
            const double cr = c * (r_min * pow(c, (double)i));
            int64_t within = 0;
            for (int64_t e = 0; e < ns; e++) {
                const int w = (i == ORC_NLEV - 1) ? 1
                              : orc_dist2_le(q, ix->X + cand[e].id * ix->d, ix->d, cr);
                if (w < 0) { bad = 1; break; }
                within += w;
            }
            if (bad) break;
            if (within >= k) { js = i; is = -1; }
        }
    }
    free(hits.v);
    free(mark);
    if (bad) { free(cand); return -2; }
    qsort(cand, (size_t)ns, sizeof(orc_cand), orc_cmp_cand);
    for (int i = 0; i < k; i++) {
        ids[i] = i < ns ? cand[i].id : -1;
        dists[i] = i < ns ? cand[i].dist : INFINITY;
    }
    if (S_size) *S_size = ns;
    if (jstop) *jstop = js;
    if (istop) *istop = is;
    free(cand);
    return 0;
}

static int orc_cmp_float_asc(const void *a, const void *b) {
    float x = *(const float *)a, y = *(const float *)b;
    return (x > y) - (x < y);
}

/* Alg. 5 at the smallest continuous r_min: every point's smallest lower bound
 * over the trees, m(o) = min_t LB^2_t(leaf_t(o)); the threshold v* is the
 * (beta*n + k)-th smallest m(o), the least squared radius (eps r)^2 at which
 * the union of the L range queries holds beta*n + k points.  Then the loop of
 * Alg. 5 at that radius: trees in order, leaves with LB^2 <= v* in ascending
 * (LB^2, leaf id) order, the check after each leaf.  eps and c cancel: only
 * the order of the lower bounds matters.  *vstar = v* (+inf when beta*n+k > n,
 * S = every point). */
int orc_index_query_magic_min(const orc_index *ix, const float *q, int k, double beta,
                              int64_t *ids, double *dists, int64_t *S_out, int64_t *S_size,
                              float *vstar, int *istar) {
    int64_t n = ix->n;
    if (k < 1 || k > n) return -1;
    int64_t tau = (int64_t)ceil(beta * (double)n) + k;
    orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)n);
    int64_t ns = 0;
    int is = -1;
    float vs = INFINITY;
    if (tau > n) {
        for (int64_t p = 0; p < n; p++) { cand[ns].id = p; if (S_out) S_out[ns] = p; ns++; }
    } else {
        float qproj[256];
        orc_query_proj(ix, q, qproj);
        float *mo = (float *)malloc(sizeof(float) * (size_t)n);
        for (int64_t p = 0; p < n; p++) mo[p] = INFINITY;
        for (int t = 0; t < ix->L; t++) {
            const otree *tr = &ix->trees[t];
            for (int64_t l = 0; l < tr->nleaves; l++) {
                const onode *lf = tr->leaves[l];
                float lb = orc_lb2(ix, t, qproj + t * ix->K, lf->lo, lf->hi);
                for (int64_t i = 0; i < lf->cnt; i++)
                    if (lb < mo[lf->ids[i]]) mo[lf->ids[i]] = lb;
            }
        }
        qsort(mo, (size_t)n, sizeof(float), orc_cmp_float_asc);
        vs = mo[tau - 1];
        free(mo);
        uint8_t *mark = (uint8_t *)calloc((size_t)n, 1);
        orc_hits hits = {0};
        for (int t = 0; t < ix->L && ns < tau; t++) {
            orc_range_query(ix, t, qproj + t * ix->K, vs, &hits);
            qsort(hits.v, (size_t)hits.n, sizeof(orc_hit), orc_cmp_hit);
            for (int64_t h = 0; h < hits.n && ns < tau; h++) {
                const onode *lf = hits.v[h].leaf;
                for (int64_t i = 0; i < lf->cnt; i++) {
                    int64_t p = lf->ids[i];
                    if (!mark[p]) {
                        mark[p] = 1;
                        if (S_out) S_out[ns] = p;
                        cand[ns++].id = p;
                    }
                }
                if (ns >= tau) is = t;
            }
        }
        free(hits.v);
        free(mark);
    }
    for (int64_t i = 0; i < ns; i++)
        cand[i].dist = orc_dist(q, ix->X + cand[i].id * ix->d, ix->d);
    qsort(cand, (size_t)ns, sizeof(orc_cand), orc_cmp_cand);
    for (int i = 0; i < k; i++) { ids[i] = cand[i].id; dists[i] = cand[i].dist; }
    if (S_size) *S_size = ns;
    if (vstar) *vstar = vs;
    if (istar) *istar = is;
    free(cand);
    return 0;
}

int orc_index_query_batch(const orc_index *ix, const float *Q, int64_t m, int k, double beta,
                          double c, int64_t *ids, double *dists, int64_t *S_sizes,
                          int nthreads) {
    int bad = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#endif
    #pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(| : bad)
    for (int64_t i = 0; i < m; i++) {
        int64_t ssz = 0;
        int rc = orc_index_query(ix, Q + i * ix->d, k, beta, c, ids + i * k, dists + i * k,
                                 NULL, &ssz, NULL, NULL);
        if (S_sizes) S_sizes[i] = ssz;
        bad |= (rc != 0);
    }
    (void)nthreads;
    return bad ? -1 : 0;
}

void orc_index_leaf_lb2(const orc_index *ix, int t, const float *q, float *lb2) {
    float qproj[16];
    for (int j = 0; j < ix->K; j++)
        qproj[j] = orc_dot_rn32(ix->A + (int64_t)(t * ix->K + j) * ix->d, q, ix->d);
    const otree *T = &ix->trees[t];
    for (int64_t l = 0; l < T->nleaves; l++)
        lb2[l] = orc_lb2(ix, t, qproj, T->leaves[l]->lo, T->leaves[l]->hi);
}

void orc_bruteforce_knn(const float *X, int64_t n, int64_t d, const float *Q, int64_t m,
                        int k, int64_t *ids, double *dists, int nthreads) {
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#endif
    #pragma omp parallel num_threads(nthreads)
    {
        orc_cand *cand = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)n);
        #pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < m; i++) {
            for (int64_t p = 0; p < n; p++) {
                cand[p].id = p;
                cand[p].dist = orc_dist(Q + i * d, X + p * d, d);
            }
            qsort(cand, (size_t)n, sizeof(orc_cand), orc_cmp_cand);
            for (int j = 0; j < k; j++) {
                ids[i * k + j] = cand[j].id;
                dists[i * k + j] = cand[j].dist;
            }
        }
        free(cand);
    }
    (void)nthreads;
}
