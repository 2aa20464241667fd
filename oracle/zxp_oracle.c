/*
 * zxp_oracle.c -- plain, slow, exact CPU oracle.  TEST INFRASTRUCTURE ONLY:
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this file's library.  It shares no code with the CUDA library.
 *
 * What it computes (Sutcliffe & Kissinger, "Fast Classical Simulation of
 * Quantum Circuits via Parametric Rewriting in the ZX-Calculus"):
 *
 *  1. oracle_ps_sum: the exponential sum of a parametric scalar, Eq. 2,
 *       S = G / sqrt2^e0 * sum_x prod_j S_j(x),
 *     over parameter assignments x = gray(t) for t in [first, first+count).
 *     Every term is evaluated on its own, from scratch, with the subterm
 *     steps of Sec. 3.3 (AND with the bits, XOR-reduce, 4x + 4alpha/pi mod 8,
 *     look up e^{i pi a/4}, combine) and the exact complex arithmetic of
 *     App. E (Lemma 5 sum, Lemma 6 product) in the paper's number form
 *     A + B sqrt2 + i (C + D sqrt2).  The four subterm kinds are the ones of
 *     App. C: node (1 + e^{i Psi}), phase-pair (Eq. 3), pi-pair
 *     (e^{i Psi Phi/pi}, used both for the linear phase terms with a fixed
 *     Psi and for the quadratic terms with two parametric phases).
 *  2. oracle_rows_eval: the row table of Sec. 3.3 / App. D (dummy flag,
 *     4alpha/pi, psi bits, 4beta/pi, phi bits), terms with constants C_i,
 *     evaluated for one parameter bitstring (Eq. 2 with phase-pair rows).
 *  3. oracle_amp / oracle_marginal: the plain definition of an amplitude
 *     <out|C|in> (Sec. 2.2), an exact state vector in Z[w]/sqrt2^e built gate
 *     by gate from the gate matrices (w = e^{i pi/4}).
 *
 * Number format.  The paper's A + B sqrt2 + i(C + D sqrt2) has A, C integers
 * and B, D half-integers for the elements used here, so every component is
 * stored doubled (2A, 2B, 2C, 2D) in signed 128-bit integers.  Every
 * operation checks for 128-bit overflow and sets a sticky flag instead of
 * wrapping.  Results are returned in the integer basis {1, w, w^2, w^3}:
 *   A + B sqrt2 + i(C + D sqrt2) = A + (B+D) w + C w^2 + (D-B) w^3.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

/* ------------------------------------------------------------------------ */
/* checked 128-bit arithmetic                                                */
/* ------------------------------------------------------------------------ */

static i128 add_c(i128 a, i128 b, int *ovf) {
    i128 r;
    if (__builtin_add_overflow(a, b, &r)) *ovf = 1;
    return r;
}
static i128 sub_c(i128 a, i128 b, int *ovf) {
    i128 r;
    if (__builtin_sub_overflow(a, b, &r)) *ovf = 1;
    return r;
}
static i128 mul_c(i128 a, i128 b, int *ovf) {
    i128 r;
    if (__builtin_mul_overflow(a, b, &r)) *ovf = 1;
    return r;
}

/* ------------------------------------------------------------------------ */
/* the paper's number form, doubled: h = (2A, 2B, 2C, 2D)                    */
/* ------------------------------------------------------------------------ */

typedef struct { i128 A2, B2, C2, D2; } abcd;

static abcd abcd_one(void) { abcd r = {2, 0, 0, 0}; return r; }
static abcd abcd_zero(void) { abcd r = {0, 0, 0, 0}; return r; }

/* Lemma 5: the sum adds like components. */
static abcd abcd_add(abcd p, abcd q, int *ovf) {
    abcd r;
    r.A2 = add_c(p.A2, q.A2, ovf);
    r.B2 = add_c(p.B2, q.B2, ovf);
    r.C2 = add_c(p.C2, q.C2, ovf);
    r.D2 = add_c(p.D2, q.D2, ovf);
    return r;
}
static abcd abcd_neg(abcd p) { abcd r = {-p.A2, -p.B2, -p.C2, -p.D2}; return r; }

/* Lemma 6: the product, written for doubled components:
 *   2A = (a1 a2 + 2 b1 b2 - c1 c2 - 2 d1 d2) / 2, and likewise for B, C, D,
 * where a1 = 2A_psi, ... .  The division is exact for elements of Z[w]. */
static abcd abcd_mul(abcd p, abcd q, int *ovf) {
    i128 a = sub_c(sub_c(add_c(mul_c(p.A2, q.A2, ovf), mul_c(2, mul_c(p.B2, q.B2, ovf), ovf), ovf),
                         mul_c(p.C2, q.C2, ovf), ovf),
                   mul_c(2, mul_c(p.D2, q.D2, ovf), ovf), ovf);
    i128 b = sub_c(sub_c(add_c(mul_c(p.A2, q.B2, ovf), mul_c(p.B2, q.A2, ovf), ovf),
                         mul_c(p.C2, q.D2, ovf), ovf),
                   mul_c(p.D2, q.C2, ovf), ovf);
    i128 c = add_c(add_c(add_c(mul_c(p.A2, q.C2, ovf), mul_c(2, mul_c(p.B2, q.D2, ovf), ovf), ovf),
                         mul_c(p.C2, q.A2, ovf), ovf),
                   mul_c(2, mul_c(p.D2, q.B2, ovf), ovf), ovf);
    i128 d = add_c(add_c(add_c(mul_c(p.A2, q.D2, ovf), mul_c(p.B2, q.C2, ovf), ovf),
                         mul_c(p.C2, q.B2, ovf), ovf),
                   mul_c(p.D2, q.A2, ovf), ovf);
    abcd r;
    /* each of a, b, c, d is even for a product of elements of Z[w] */
    if ((a & 1) || (b & 1) || (c & 1) || (d & 1)) *ovf = 1;
    r.A2 = a / 2; r.B2 = b / 2; r.C2 = c / 2; r.D2 = d / 2;
    return r;
}

/* Sec. 3.3 step 4: look-up table e^{i pi a/4} -> A + B sqrt2 + i(C + D sqrt2),
 * a in 0..7 (cos/sin of multiples of pi/4 are 0, +-1, +-sqrt2/2). */
static abcd lut_exp(unsigned a) {
    static const int T[8][4] = {
        { 2,  0,  0,  0},   /* 1                          */
        { 0,  1,  0,  1},   /* sqrt2/2 + i sqrt2/2        */
        { 0,  0,  2,  0},   /* i                          */
        { 0, -1,  0,  1},   /* -sqrt2/2 + i sqrt2/2       */
        {-2,  0,  0,  0},   /* -1                         */
        { 0, -1,  0, -1},   /* -sqrt2/2 - i sqrt2/2       */
        { 0,  0, -2,  0},   /* -i                         */
        { 0,  1,  0, -1},   /* sqrt2/2 - i sqrt2/2        */
    };
    abcd r = {T[a & 7][0], T[a & 7][1], T[a & 7][2], T[a & 7][3]};
    return r;
}

/* A + B sqrt2 + i(C + D sqrt2) = A + (B+D) w + C w^2 + (D-B) w^3 */
static void abcd_to_omega(abcd p, i128 c[4], int *ovf) {
    i128 bd = add_c(p.B2, p.D2, ovf), db = sub_c(p.D2, p.B2, ovf);
    if ((p.A2 & 1) || (p.C2 & 1) || (bd & 1) || (db & 1)) *ovf = 1;
    c[0] = p.A2 / 2; c[1] = bd / 2; c[2] = p.C2 / 2; c[3] = db / 2;
}

/* inverse: w = sqrt2/2 (1+i), w^3 = sqrt2/2 (-1+i) */
static abcd omega_to_abcd(const int64_t c[4]) {
    abcd r;
    r.A2 = 2 * (i128)c[0];
    r.B2 = (i128)c[1] - (i128)c[3];
    r.C2 = 2 * (i128)c[2];
    r.D2 = (i128)c[1] + (i128)c[3];
    return r;
}

/* ------------------------------------------------------------------------ */
/* subterms (App. C table; Sec. 3.3 steps 1-6)                               */
/* ------------------------------------------------------------------------ */

/* steps 2-3: AND the row's bits with the parameter bits, XOR-reduce */
static unsigned parity_of(uint64_t mask, uint64_t bits) {
    uint64_t v = mask & bits;
    unsigned p = 0;
    while (v) { p ^= 1u; v &= v - 1; }
    return p;
}

/* Phase-pair, Eq. 3: s = 1 + e^{i Psi} + e^{i Phi} - e^{i (Psi + Phi)}, with
 * 4Psi/pi = 4x + a mod 8 and 4Phi/pi = 4y + b mod 8 (steps 2-6). */
static abcd phase_pair(unsigned a, uint64_t psi_mask, unsigned b, uint64_t phi_mask,
                       uint64_t bits, int *ovf) {
    unsigned x = parity_of(psi_mask, bits);                /* steps 2-3 */
    unsigned y = parity_of(phi_mask, bits);
    unsigned psi4 = (4 * x + a) % 8, phi4 = (4 * y + b) % 8; /* step 4 */
    abcd e_psi = lut_exp(psi4), e_phi = lut_exp(phi4);     /* step 5 */
    abcd e_sum = lut_exp((psi4 + phi4) % 8);
    abcd s = abcd_add(abcd_add(abcd_one(), e_psi, ovf), e_phi, ovf);  /* step 6 */
    return abcd_add(s, abcd_neg(e_sum), ovf);
}

/* Node: 1 + e^{i Psi}, 4Psi/pi = 4x + a mod 8. */
static abcd node_term(unsigned a, uint64_t mask, uint64_t bits, int *ovf) {
    unsigned x = parity_of(mask, bits);
    return abcd_add(abcd_one(), lut_exp((4 * x + a) % 8), ovf);
}

/* pi-pair: e^{i Psi Phi / pi}.  Psi = pi lA, Phi = pi lB for a quadratic
 * term (so Psi Phi / pi = pi lA lB); Psi = c pi/4 fixed, Phi = pi l for a
 * linear term (so Psi Phi / pi = c l pi/4). */
static abcd pi_pair_quadratic(uint64_t ma, uint64_t mb, uint64_t bits) {
    return lut_exp(4 * (parity_of(ma, bits) & parity_of(mb, bits)));
}
static abcd pi_pair_linear(unsigned c, uint64_t mask, uint64_t bits) {
    return lut_exp((c * parity_of(mask, bits)) % 8);
}

/* ------------------------------------------------------------------------ */
/* canonical form (c0..c3)/sqrt2^e in the basis {1, w, w^2, w^3}             */
/* ------------------------------------------------------------------------ */

/* x sqrt2 = (c1 - c3) + (c0 + c2) w + (c1 + c3) w^2 + (c2 - c0) w^3; x is a
 * multiple of sqrt2 iff c0 = c2 and c1 = c3 mod 2, and then x / sqrt2 is half
 * of x sqrt2. */
static void canon(i128 c[4], int32_t *e, int *ovf) {
    if (c[0] == 0 && c[1] == 0 && c[2] == 0 && c[3] == 0) { *e = 0; return; }
    while (*e > 0 && ((c[0] - c[2]) & 1) == 0 && ((c[1] - c[3]) & 1) == 0) {
        i128 n0 = sub_c(c[1], c[3], ovf), n1 = add_c(c[0], c[2], ovf);
        i128 n2 = add_c(c[1], c[3], ovf), n3 = sub_c(c[2], c[0], ovf);
        c[0] = n0 / 2; c[1] = n1 / 2; c[2] = n2 / 2; c[3] = n3 / 2;
        *e -= 1;
    }
}

static void omega_mul(i128 r[4], const i128 p[4], const i128 q[4], int *ovf) {
    /* (sum p_i w^i)(sum q_j w^j) with w^4 = -1 */
    i128 t[4] = {0, 0, 0, 0};
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            i128 m = mul_c(p[i], q[j], ovf);
            int s = i + j;
            if (s < 4) t[s] = add_c(t[s], m, ovf);
            else t[s - 4] = sub_c(t[s - 4], m, ovf);
        }
    memcpy(r, t, sizeof t);
}

/* ------------------------------------------------------------------------ */
/* parametric-scalar table blob (layout shared with the generator module)    */
/* ------------------------------------------------------------------------ */

#define PS_MAGIC 0x5350585Au
typedef struct {
    uint32_t magic, version, k, n_lin, n_quad, n_node, n_pair;
    int32_t e0;
    int64_t G[4];
} ps_header;

/* Version 2 appends {u32 k_inner, u32 0} to the header: the last k_inner
 * of the k parameters are inner ones.  The value is the same Eq. 2 sum over
 * all 2^k assignments; only the indexing of terms changes (see
 * oracle_ps_sum). */
typedef struct {
    ps_header h;
    uint32_t k_inner;
    const uint8_t *lin, *quad, *node, *pair;
} ps_view;

static int ps_parse(const void *blob, size_t nbytes, ps_view *v) {
    if (nbytes < sizeof(ps_header)) return -1;
    memcpy(&v->h, blob, sizeof(ps_header));
    if (v->h.magic != PS_MAGIC || (v->h.version != 1 && v->h.version != 2) || v->h.k > 62) return -1;
    size_t hsize = sizeof(ps_header) + (v->h.version == 2 ? 8u : 0u);
    v->k_inner = 0;
    if (v->h.version == 2) {
        if (nbytes < hsize) return -1;
        memcpy(&v->k_inner, (const uint8_t *)blob + sizeof(ps_header), 4);
        if (v->k_inner > v->h.k) return -1;
    }
    size_t need = hsize + 16u * v->h.n_lin + 16u * v->h.n_quad +
                  16u * v->h.n_node + 24u * v->h.n_pair;
    if (nbytes < need) return -1;
    const uint8_t *p = (const uint8_t *)blob + hsize;
    v->lin = p;  p += 16u * v->h.n_lin;
    v->quad = p; p += 16u * v->h.n_quad;
    v->node = p; p += 16u * v->h.n_node;
    v->pair = p;
    return 0;
}
static uint64_t rd64(const uint8_t *p) { uint64_t v; memcpy(&v, p, 8); return v; }
static uint32_t rd32(const uint8_t *p) { uint32_t v; memcpy(&v, p, 4); return v; }

/* One term of Eq. 2 at parameter bits x: the product of every subterm. */
static abcd ps_term(const ps_view *v, uint64_t x, int *ovf) {
    abcd t = abcd_one();
    for (uint32_t j = 0; j < v->h.n_lin; j++) {
        const uint8_t *r = v->lin + 16u * j;
        t = abcd_mul(t, pi_pair_linear(rd32(r + 8) & 7, rd64(r), x), ovf);
    }
    for (uint32_t j = 0; j < v->h.n_quad; j++) {
        const uint8_t *r = v->quad + 16u * j;
        t = abcd_mul(t, pi_pair_quadratic(rd64(r), rd64(r + 8), x), ovf);
    }
    for (uint32_t j = 0; j < v->h.n_node; j++) {
        const uint8_t *r = v->node + 16u * j;
        t = abcd_mul(t, node_term(rd32(r + 8) & 7, rd64(r), x, ovf), ovf);
    }
    for (uint32_t j = 0; j < v->h.n_pair; j++) {
        const uint8_t *r = v->pair + 24u * j;
        t = abcd_mul(t, phase_pair(rd32(r + 16) & 7, rd64(r), rd32(r + 20) & 7,
                                   rd64(r + 8), x, ovf), ovf);
    }
    return t;
}

/* Sum of the terms for Gray-code indices t in [first, first + count) (the
 * term of index t is the assignment x = t xor (t >> 1)), multiplied by G.
 * With k_inner > 0 (version 2 tables) the index t runs over the first
 * k_o = k - k_inner parameters only, and the term of index t is the sum of
 * Eq. 2's terms over every value y of the inner parameters:
 * x = gray(t) | (y << k_o), y in [0, 2^k_inner).  Over the whole range
 * [0, 2^k_o) this is again the sum over all 2^k assignments.
 * out_c[8] = four signed 128-bit coefficients as (lo, hi) uint64 pairs,
 * in the basis {1, w, w^2, w^3}, over sqrt2^e0 (not reduced).
 * Returns 0, -1 for a bad blob or range, 1 if a 128-bit overflow occurred.
 * nthreads > 1 splits the index range into contiguous pieces whose exact
 * integer sums are added at the end. */
int oracle_ps_sum(const void *blob, size_t nbytes, uint64_t first, uint64_t count,
                  int nthreads, uint64_t out_c[8], int32_t *out_e) {
    ps_view v;
    if (ps_parse(blob, nbytes, &v) != 0) return -1;
    const uint32_t k_o = v.h.k - v.k_inner;
    const uint64_t total = (uint64_t)1 << k_o, n_inner = (uint64_t)1 << v.k_inner;
    if (first > total || count > total - first) return -1;
    if (count && n_inner > UINT64_MAX / count) return -1;   /* more terms than any run could take */
    const uint64_t flat = count * n_inner;
    if (nthreads < 1) nthreads = 1;
    abcd *part = (abcd *)calloc((size_t)nthreads, sizeof(abcd));
    int *povf = (int *)calloc((size_t)nthreads, sizeof(int));
    if (!part || !povf) { free(part); free(povf); return -1; }
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int tid = 0, nt = 1;
#ifdef _OPENMP
        tid = omp_get_thread_num(); nt = omp_get_num_threads();
#endif
        /* each thread takes a contiguous piece of the (term, inner value)
         * pairs f = (t - first) * n_inner + y */
        uint64_t ut = (uint64_t)tid, rem = flat % (uint64_t)nt;
        uint64_t lo = (flat / (uint64_t)nt) * ut + (ut < rem ? ut : rem);
        uint64_t len = flat / (uint64_t)nt + (ut < rem ? 1 : 0);
        uint64_t t = first + lo / n_inner, y = lo % n_inner;
        abcd s = abcd_zero();
        int ovf = 0;
        for (uint64_t f = 0; f < len; f++) {
            uint64_t x = t ^ (t >> 1);
            s = abcd_add(s, ps_term(&v, x | (y << k_o), &ovf), &ovf);
            if (++y == n_inner) { y = 0; t++; }
        }
        part[tid] = s; povf[tid] = ovf;
    }
    abcd s = abcd_zero();
    int ovf = 0;
    for (int i = 0; i < nthreads; i++) { s = abcd_add(s, part[i], &ovf); ovf |= povf[i]; }
    free(part); free(povf);
    /* multiply by the global constant G */
    s = abcd_mul(s, omega_to_abcd(v.h.G), &ovf);
    i128 c[4];
    abcd_to_omega(s, c, &ovf);
    for (int i = 0; i < 4; i++) { out_c[2 * i] = (uint64_t)c[i]; out_c[2 * i + 1] = (uint64_t)(c[i] >> 64); }
    *out_e = v.h.e0;
    return ovf ? 1 : 0;
}

/* Value of a single term (no G): for brute-force checks. */
int oracle_ps_term(const void *blob, size_t nbytes, uint64_t x, uint64_t out_c[8]) {
    ps_view v;
    if (ps_parse(blob, nbytes, &v) != 0) return -1;
    int ovf = 0;
    abcd t = ps_term(&v, x, &ovf);
    i128 c[4];
    abcd_to_omega(t, c, &ovf);
    for (int i = 0; i < 4; i++) { out_c[2 * i] = (uint64_t)c[i]; out_c[2 * i + 1] = (uint64_t)(c[i] >> 64); }
    return ovf ? 1 : 0;
}

/* Canonical form of a 128-bit numerator over sqrt2^e. */
int oracle_canon(const uint64_t in_c[8], int32_t e, uint64_t out_c[8], int32_t *out_e) {
    i128 c[4];
    int ovf = 0;
    for (int i = 0; i < 4; i++) c[i] = (i128)(((unsigned __int128)in_c[2 * i + 1] << 64) | in_c[2 * i]);
    canon(c, &e, &ovf);
    for (int i = 0; i < 4; i++) { out_c[2 * i] = (uint64_t)c[i]; out_c[2 * i + 1] = (uint64_t)(c[i] >> 64); }
    *out_e = e;
    return ovf ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* the row table of Sec. 3.3 / App. D                                         */
/* ------------------------------------------------------------------------ */

/* rows[r] = {star, a, psi_mask, b, phi_mask}; terms are consecutive groups of
 * rows_per_term rows; C[i] = constant of term i in the basis {1,w,w^2,w^3}.
 * S(p) = sum_i C_i prod_j S_ij(p), dummy rows (star = 0) giving 1 (step 1). */
int oracle_rows_eval(const uint64_t *rows, uint32_t n_terms, uint32_t rows_per_term,
                     const int64_t *C, uint64_t p, uint64_t out_c[8]) {
    int ovf = 0;
    abcd S = abcd_zero();
    for (uint32_t i = 0; i < n_terms; i++) {
        abcd prod = abcd_one();
        for (uint32_t j = 0; j < rows_per_term; j++) {
            const uint64_t *r = rows + 5u * (i * rows_per_term + j);
            abcd s = r[0] ? phase_pair((unsigned)r[1] & 7, r[2], (unsigned)r[3] & 7, r[4], p, &ovf)
                          : abcd_one();
            prod = abcd_mul(prod, s, &ovf);
        }
        S = abcd_add(S, abcd_mul(omega_to_abcd(C + 4 * i), prod, &ovf), &ovf);
    }
    i128 c[4];
    abcd_to_omega(S, c, &ovf);
    for (int i = 0; i < 4; i++) { out_c[2 * i] = (uint64_t)c[i]; out_c[2 * i + 1] = (uint64_t)(c[i] >> 64); }
    return ovf ? 1 : 0;
}

/* Exported single-operation hooks so that tests can pin the arithmetic
 * (Lemma 5, Lemma 6, the look-up table) against complex floating point. */
void oracle_abcd_lut(unsigned a, int64_t out[4]) {
    abcd r = lut_exp(a);
    out[0] = (int64_t)r.A2; out[1] = (int64_t)r.B2; out[2] = (int64_t)r.C2; out[3] = (int64_t)r.D2;
}
int oracle_abcd_mul(const int64_t p[4], const int64_t q[4], int64_t out[4]) {
    int ovf = 0;
    abcd a = {p[0], p[1], p[2], p[3]}, b = {q[0], q[1], q[2], q[3]};
    abcd r = abcd_mul(a, b, &ovf);
    out[0] = (int64_t)r.A2; out[1] = (int64_t)r.B2; out[2] = (int64_t)r.C2; out[3] = (int64_t)r.D2;
    return ovf;
}
int oracle_abcd_add(const int64_t p[4], const int64_t q[4], int64_t out[4]) {
    int ovf = 0;
    abcd a = {p[0], p[1], p[2], p[3]}, b = {q[0], q[1], q[2], q[3]};
    abcd r = abcd_add(a, b, &ovf);
    out[0] = (int64_t)r.A2; out[1] = (int64_t)r.B2; out[2] = (int64_t)r.C2; out[3] = (int64_t)r.D2;
    return ovf;
}
/* Subterm values for every (x, y) in {0,1}^2 (pins of Eq. 3 / App. C). */
int oracle_subterm(int kind, unsigned a, unsigned b, unsigned x, unsigned y, int64_t out_w[4]) {
    int ovf = 0;
    abcd s;
    switch (kind) {
    case 0: s = node_term(a, 1, x, &ovf); break;                     /* node */
    case 1: s = phase_pair(a, 1, b, 2, (uint64_t)x | ((uint64_t)y << 1), &ovf); break;
    case 2: s = pi_pair_quadratic(1, 2, (uint64_t)x | ((uint64_t)y << 1)); break;
    case 3: s = pi_pair_linear(a, 1, x); break;
    default: return -1;
    }
    i128 c[4];
    abcd_to_omega(s, c, &ovf);
    for (int i = 0; i < 4; i++) out_w[i] = (int64_t)c[i];
    return ovf;
}

/* ------------------------------------------------------------------------ */
/* exact state vector (Sec. 2.2: amplitude of a closed diagram)              */
/* ------------------------------------------------------------------------ */

enum { G_H = 0, G_S, G_T, G_CNOT, G_SDG, G_TDG, G_X, G_Z, G_CZ };
typedef struct { uint8_t op, r; uint16_t q0, q1, r2; } gate_rec;

typedef struct { i128 c[4]; } zw;   /* c0 + c1 w + c2 w^2 + c3 w^3 */

static zw zw_rot(zw a, int j) {       /* a * w^j */
    zw r = a;
    for (int s = 0; s < (j & 7); s++) {
        zw t = {{-r.c[3], r.c[0], r.c[1], r.c[2]}};
        r = t;
    }
    return r;
}

typedef struct { zw *v; uint64_t dim; int32_t e; int ovf; } svec;

static int sv_apply(svec *s, int n, const gate_rec *g) {
    uint64_t dim = s->dim;
    unsigned op = g->op, q0 = g->q0, q1 = g->q1;
    if (q0 >= (unsigned)n) return -1;
    if ((op == G_CNOT || op == G_CZ) && (q1 >= (unsigned)n || q1 == q0)) return -1;
    uint64_t b0 = (uint64_t)1 << q0, b1 = (op == G_CNOT || op == G_CZ) ? (uint64_t)1 << q1 : 0;
    switch (op) {
    case G_H:          /* H = (1/sqrt2) [[1, 1], [1, -1]] */
        for (uint64_t i = 0; i < dim; i++)
            if (!(i & b0)) {
                zw a = s->v[i], b = s->v[i | b0];
                for (int j = 0; j < 4; j++) {
                    s->v[i].c[j] = add_c(a.c[j], b.c[j], &s->ovf);
                    s->v[i | b0].c[j] = sub_c(a.c[j], b.c[j], &s->ovf);
                }
            }
        s->e += 1;
        break;
    case G_S: case G_T: case G_SDG: case G_TDG: case G_Z: {
        int j = op == G_S ? 2 : op == G_T ? 1 : op == G_SDG ? 6 : op == G_TDG ? 7 : 4;
        for (uint64_t i = 0; i < dim; i++) if (i & b0) s->v[i] = zw_rot(s->v[i], j);
        break;
    }
    case G_X:
        for (uint64_t i = 0; i < dim; i++)
            if (!(i & b0)) { zw t = s->v[i]; s->v[i] = s->v[i | b0]; s->v[i | b0] = t; }
        break;
    case G_CNOT:       /* control q0, target q1 */
        for (uint64_t i = 0; i < dim; i++)
            if ((i & b0) && !(i & b1)) { zw t = s->v[i]; s->v[i] = s->v[i | b1]; s->v[i | b1] = t; }
        break;
    case G_CZ:
        for (uint64_t i = 0; i < dim; i++) if ((i & b0) && (i & b1)) s->v[i] = zw_rot(s->v[i], 4);
        break;
    default:
        return -1;
    }
    return 0;
}

/* divide the whole vector by sqrt2 while every entry allows it */
static void sv_reduce(svec *s) {
    while (s->e > 0) {
        for (uint64_t i = 0; i < s->dim; i++) {
            i128 *c = s->v[i].c;
            if (((c[0] - c[2]) & 1) || ((c[1] - c[3]) & 1)) return;
        }
        for (uint64_t i = 0; i < s->dim; i++) {
            i128 *c = s->v[i].c;
            i128 n0 = c[1] - c[3], n1 = c[0] + c[2], n2 = c[1] + c[3], n3 = c[2] - c[0];
            c[0] = n0 / 2; c[1] = n1 / 2; c[2] = n2 / 2; c[3] = n3 / 2;
        }
        s->e -= 1;
    }
}

static int sv_run(svec *s, const void *gates, size_t ng, int n, const uint8_t *in_bits) {
    if (n < 1 || n > 26) return -1;
    s->dim = (uint64_t)1 << n;
    s->v = (zw *)calloc(s->dim, sizeof(zw));
    if (!s->v) return -1;
    s->e = 0; s->ovf = 0;
    uint64_t idx0 = 0;
    for (int q = 0; q < n; q++) if (in_bits && in_bits[q]) idx0 |= (uint64_t)1 << q;
    s->v[idx0].c[0] = 1;
    const gate_rec *g = (const gate_rec *)gates;
    for (size_t i = 0; i < ng; i++) {
        if (sv_apply(s, n, &g[i]) != 0) { free(s->v); s->v = NULL; return -1; }
        if (g[i].op == G_H) sv_reduce(s);
    }
    return 0;
}

/* <out|C|in>, canonical, qubit q <-> bit q of the basis index. */
int oracle_amp(const void *gates, size_t ng, int n, const uint8_t *in_bits,
               const uint8_t *out_bits, uint64_t out_c[8], int32_t *out_e) {
    svec s;
    if (sv_run(&s, gates, ng, n, in_bits) != 0) return -1;
    uint64_t idx = 0;
    for (int q = 0; q < n; q++) if (out_bits[q]) idx |= (uint64_t)1 << q;
    i128 c[4];
    memcpy(c, s.v[idx].c, sizeof c);
    int32_t e = s.e;
    int ovf = s.ovf;
    free(s.v);
    canon(c, &e, &ovf);
    for (int i = 0; i < 4; i++) { out_c[2 * i] = (uint64_t)c[i]; out_c[2 * i + 1] = (uint64_t)(c[i] >> 64); }
    *out_e = e;
    return ovf ? 1 : 0;
}

/* Every amplitude <x|C|in> for x in [0, 2^n): out[8*x..] as in oracle_amp,
 * e_out[x] their exponents (canonical). */
int oracle_amps_all(const void *gates, size_t ng, int n, const uint8_t *in_bits,
                    uint64_t *out_c, int32_t *out_e) {
    svec s;
    if (sv_run(&s, gates, ng, n, in_bits) != 0) return -1;
    int ovf = s.ovf;
    for (uint64_t x = 0; x < s.dim; x++) {
        i128 c[4];
        memcpy(c, s.v[x].c, sizeof c);
        int32_t e = s.e;
        canon(c, &e, &ovf);
        for (int i = 0; i < 4; i++) {
            out_c[8 * x + 2 * i] = (uint64_t)c[i];
            out_c[8 * x + 2 * i + 1] = (uint64_t)(c[i] >> 64);
        }
        out_e[x] = e;
    }
    free(s.v);
    return ovf ? 1 : 0;
}

/* Marginal probability P(q = bits[q] for every q in mask) of C|in>
 * (Sec. 2.2, Born rule): the sum of |amp|^2 over the unfixed qubits.
 * |z|^2 = z * conj(z), conj(sum c_j w^j) = c0 - c3 w - c2 w^2 - c1 w^3. */
int oracle_marginal(const void *gates, size_t ng, int n, const uint8_t *in_bits,
                    uint64_t mask, const uint8_t *bits, uint64_t out_c[8], int32_t *out_e) {
    svec s;
    if (sv_run(&s, gates, ng, n, in_bits) != 0) return -1;
    uint64_t want = 0;
    for (int q = 0; q < n; q++) if (bits[q]) want |= (uint64_t)1 << q;
    want &= mask;
    i128 acc[4] = {0, 0, 0, 0};
    int ovf = s.ovf;
    for (uint64_t x = 0; x < s.dim; x++) {
        if ((x & mask) != want) continue;
        i128 *c = s.v[x].c;
        i128 cj[4] = {c[0], -c[3], -c[2], -c[1]};
        i128 m[4];
        omega_mul(m, c, cj, &ovf);
        for (int i = 0; i < 4; i++) acc[i] = add_c(acc[i], m[i], &ovf);
    }
    int32_t e = 2 * s.e;
    free(s.v);
    canon(acc, &e, &ovf);
    for (int i = 0; i < 4; i++) { out_c[2 * i] = (uint64_t)acc[i]; out_c[2 * i + 1] = (uint64_t)(acc[i] >> 64); }
    *out_e = e;
    return ovf ? 1 : 0;
}
