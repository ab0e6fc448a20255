/*
 * oracle.c -- plain, slow, CPU FP64 reference for compressed state-vector
 * simulation (MEMQSim, arXiv 2309.16979).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's
 * CPU-baseline leg load this library; the product path never calls it and
 * shares no code with it.
 *
 * What it computes, and where each part comes from:
 *   1. Gate matrices: textbook definitions (H, Paulis, S, T, rotations
 *      U = exp(-i theta G / 2), phase, controlled forms, SWAP, custom).
 *   2. psi <- U psi for one gate at a time on a full complex128 state
 *      (Sec. 2: the GPU "updates the state vector amplitudes"; here an
 *      unblocked loop over every amplitude, no chunking, no compression).
 *   3. <psi| sum_j c_j P_j |psi> for Pauli strings P_j.
 *   4. Gradients of E(theta) = <psi(theta)|H|psi(theta)>: the adjoint
 *      recursion of Jones & Gacon (arXiv 2009.02823), g_k = Im<lambda_k|G_k|psi_k>.
 *   5. Reference codec for one chunk (Sec. 2 "Offline stage": every chunk of
 *      the state vector is compressed independently). The paper names no
 *      compressor; this is the error-bounded linear quantiser with per-block
 *      1-D Lorenzo prediction and 256-value fixed-length bit packing with
 *      prefix-sum block offsets that the library implements. Its byte stream
 *      is the format definition:
 *
 *        offset  size  field
 *        0       4     magic 0x31435653 ("SVC1", little-endian)
 *        4       2     version = 1
 *        6       1     dtype (1 = complex64, 2 = complex128)
 *        7       1     c = log2(amplitudes per chunk), 8..30
 *        8       4     int32 k, quantisation step Delta = 2^k
 *        12      4     nblocks = 2 * 2^c / 256
 *        16      4     total_words (payload length in uint32 words)
 *        20      12    zero
 *        32      ...   uint8 width[nblocks], padded to 16 bytes
 *        ...     ...   int32 anchor[nblocks], padded to 16 bytes
 *        ...     ...   uint32 offset[nblocks + 1], padded to 16 bytes
 *        ...     ...   uint32 payload[total_words]
 *
 *      Blocks 0 .. nblocks/2-1 hold the real parts (plane 0) of amplitudes
 *      256b .. 256b+255; blocks nblocks/2 .. hold the imaginary parts.
 *      Delta is the largest power of two <= 2*eb, so q*Delta is exact and
 *      |x - q*Delta| <= Delta/2 <= eb holds exactly.
 *      Per block: q_j = rint(x_j / Delta) (ties to even); anchor = q_0;
 *      r_0 = 0, r_j = q_j - q_{j-1}; z_j = zigzag(r_j) = 2 r_j for r_j >= 0,
 *      -2 r_j - 1 otherwise; width w = bit length of max_j z_j; value j
 *      occupies bits [j*w, j*w + w) of the block's little-endian bit string
 *      of 8*w words; offset[b+1] = offset[b] + 8*w_b, offset[0] = 0.
 *      |q| must not exceed 2^24 - 1 (complex64) or 2^30 - 1 (complex128).
 *
 *      Relative bound (the paper fixes no bound; a reading that keeps spread
 *      states from quantising to zero): a chunk whose largest component
 *      magnitude is m > 0 takes k = floor(log2(2 * eb * m)) clamped to
 *      [-60, 0] (k = 0 when m = 0), so |x - q*Delta| <= max(eb * m, 2^-61)
 *      for every component. The stream format is the same; only k differs
 *      between chunks.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- types */

typedef struct { double re, im; } cx;

static cx cx_make(double re, double im) { cx z; z.re = re; z.im = im; return z; }
static cx cx_add(cx a, cx b) { return cx_make(a.re + b.re, a.im + b.im); }
static cx cx_mul(cx a, cx b) { return cx_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static cx cx_conj(cx a) { return cx_make(a.re, -a.im); }
static cx cx_scale(cx a, double s) { return cx_make(a.re * s, a.im * s); }

/* gate kinds (oracle numbering) */
enum {
    OR_H = 0, OR_X, OR_Y, OR_Z, OR_S, OR_SDG, OR_T, OR_TDG, OR_RX, OR_RY, OR_RZ,
    OR_P, OR_CNOT, OR_CZ, OR_CP, OR_SWAP, OR_CUSTOM
};

typedef struct {
    int32_t kind;
    int32_t nt;          /* number of targets (1 or 2) */
    int32_t nc;          /* number of controls (0..2) */
    int32_t param;       /* parameter index or -1 */
    int32_t t[2];
    int32_t c[2];
    double theta;
    double m[32];        /* CUSTOM: row-major 2^nt x 2^nt complex (re, im pairs) */
} or_gate;

typedef struct {
    double coeff;
    uint64_t x;
    uint64_t z;
} or_pauli;

/* status codes */
#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_CORRUPT -4
#define OR_ERR_RANGE -7

/* ------------------------------------------------------- gate matrices */

/* Fill m (2^nt x 2^nt, row-major) with the gate's target matrix. Controls are
 * handled separately: the matrix acts only where all controls are 1. */
static int gate_matrix(const or_gate *g, double theta, cx *m)
{
    const double r2 = 1.0 / sqrt(2.0);
    double c = cos(theta / 2.0), s = sin(theta / 2.0);
    int i;
    for (i = 0; i < 16; i++) m[i] = cx_make(0, 0);
    switch (g->kind) {
    case OR_H: m[0] = cx_make(r2, 0); m[1] = cx_make(r2, 0); m[2] = cx_make(r2, 0); m[3] = cx_make(-r2, 0); return 1;
    case OR_X: case OR_CNOT: m[1] = cx_make(1, 0); m[2] = cx_make(1, 0); return 1;
    case OR_Y: m[1] = cx_make(0, -1); m[2] = cx_make(0, 1); return 1;
    case OR_Z: case OR_CZ: m[0] = cx_make(1, 0); m[3] = cx_make(-1, 0); return 1;
    case OR_S: m[0] = cx_make(1, 0); m[3] = cx_make(0, 1); return 1;
    case OR_SDG: m[0] = cx_make(1, 0); m[3] = cx_make(0, -1); return 1;
    case OR_T: m[0] = cx_make(1, 0); m[3] = cx_make(r2, r2); return 1;
    case OR_TDG: m[0] = cx_make(1, 0); m[3] = cx_make(r2, -r2); return 1;
    case OR_RX: /* exp(-i theta X / 2) */
        m[0] = cx_make(c, 0); m[1] = cx_make(0, -s); m[2] = cx_make(0, -s); m[3] = cx_make(c, 0); return 1;
    case OR_RY: /* exp(-i theta Y / 2) */
        m[0] = cx_make(c, 0); m[1] = cx_make(-s, 0); m[2] = cx_make(s, 0); m[3] = cx_make(c, 0); return 1;
    case OR_RZ: /* exp(-i theta Z / 2) */
        m[0] = cx_make(c, -s); m[3] = cx_make(c, s); return 1;
    case OR_P: case OR_CP:
        m[0] = cx_make(1, 0); m[3] = cx_make(cos(theta), sin(theta)); return 1;
    case OR_SWAP:
        m[0] = cx_make(1, 0); m[6] = cx_make(1, 0); m[9] = cx_make(1, 0); m[15] = cx_make(1, 0); return 2;
    case OR_CUSTOM: {
        int k = 1 << g->nt;
        for (i = 0; i < k * k; i++) m[i] = cx_make(g->m[2 * i], g->m[2 * i + 1]);
        return g->nt;
    }
    default: return -1;
    }
}

/* ----------------------------------------------------- state updates */

/* psi <- M psi on the targets, where all controls are 1. Matrix index bit b
 * corresponds to target t[b]. Each target group is visited once, from its
 * member with all target bits 0. */
static void apply_matrix(int n, cx *psi, int nt, const int32_t *t, int nc, const int32_t *c, const cx *M)
{
    uint64_t dim = 1ULL << n, tmask = 0, cmask = 0;
    int K = 1 << nt, a, b;
    int64_t i;
    for (a = 0; a < nt; a++) tmask |= 1ULL << t[a];
    for (a = 0; a < nc; a++) cmask |= 1ULL << c[a];
#pragma omp parallel for schedule(static) private(a, b)
    for (i = 0; i < (int64_t)dim; i++) {
        uint64_t idx[4];
        cx v[4], w[4];
        if ((uint64_t)i & tmask) continue;
        if (((uint64_t)i & cmask) != cmask) continue;
        for (a = 0; a < K; a++) {
            uint64_t j = (uint64_t)i;
            for (b = 0; b < nt; b++)
                if ((a >> b) & 1) j |= 1ULL << t[b];
            idx[a] = j;
            v[a] = psi[j];
        }
        for (a = 0; a < K; a++) {
            cx acc = cx_make(0, 0);
            for (b = 0; b < K; b++) acc = cx_add(acc, cx_mul(M[a * K + b], v[b]));
            w[a] = acc;
        }
        for (a = 0; a < K; a++) psi[idx[a]] = w[a];
    }
}

static int gate_valid(int n, const or_gate *g)
{
    int a, b;
    uint64_t seen = 0;
    if (g->nt < 1 || g->nt > 2 || g->nc < 0 || g->nc > 2) return 0;
    if (g->kind == OR_SWAP && g->nt != 2) return 0;
    if ((g->kind == OR_CNOT || g->kind == OR_CZ || g->kind == OR_CP) && g->nc < 1) return 0;
    if (g->kind != OR_SWAP && g->kind != OR_CUSTOM && g->nt != 1) return 0;
    for (a = 0; a < g->nt + g->nc; a++) {
        int q = a < g->nt ? g->t[a] : g->c[a - g->nt];
        if (q < 0 || q >= n) return 0;
        if (seen & (1ULL << q)) return 0;
        seen |= 1ULL << q;
    }
    (void)b;
    return 1;
}

/* theta_override: if non-NULL and g->param >= 0, the angle is theta_override[param] */
static int apply_gate(int n, cx *psi, const or_gate *g, const double *theta_override, int dagger)
{
    cx M[16], D[16];
    double th = g->theta;
    int nt, K, a, b;
    if (!gate_valid(n, g)) return OR_ERR_ARG;
    if (theta_override && g->param >= 0) th = theta_override[g->param];
    nt = gate_matrix(g, th, M);
    if (nt < 0) return OR_ERR_ARG;
    K = 1 << nt;
    if (dagger) {
        for (a = 0; a < K; a++)
            for (b = 0; b < K; b++) D[a * K + b] = cx_conj(M[b * K + a]);
        memcpy(M, D, sizeof(cx) * K * K);
    }
    apply_matrix(n, psi, nt, g->t, g->nc, g->c, M);
    return OR_OK;
}

/* (P psi)[k] = phase(k ^ x) psi[k ^ x], with P|m> = i^{ny} (-1)^{popcount(m & z)} |m ^ x> */
static cx pauli_phase(const or_pauli *p, uint64_t m)
{
    int ny = __builtin_popcountll(p->x & p->z) & 3;
    int sign = __builtin_popcountll(m & p->z) & 1;
    cx ph;
    switch (ny) {
    case 0: ph = cx_make(1, 0); break;
    case 1: ph = cx_make(0, 1); break;
    case 2: ph = cx_make(-1, 0); break;
    default: ph = cx_make(0, -1); break;
    }
    return sign ? cx_scale(ph, -1.0) : ph;
}

/* <a| P |b> = sum_m conj(a[m ^ x]) phase(m) b[m] */
static cx pauli_braket(int n, const cx *a, const or_pauli *p, const cx *b)
{
    uint64_t dim = 1ULL << n;
    double re = 0, im = 0;
    int64_t m;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
    for (m = 0; m < (int64_t)dim; m++) {
        cx term = cx_mul(cx_conj(a[(uint64_t)m ^ p->x]), cx_mul(pauli_phase(p, (uint64_t)m), b[m]));
        re += term.re;
        im += term.im;
    }
    return cx_make(re, im);
}

/* ------------------------------------------------------------ exports */

int or_apply_gates(int n, double *psi, const or_gate *g, int64_t ng, const double *theta)
{
    int64_t i;
    if (n < 1 || n > 40) return OR_ERR_ARG;
    for (i = 0; i < ng; i++) {
        int s = apply_gate(n, (cx *)psi, &g[i], theta, 0);
        if (s) return s;
    }
    return OR_OK;
}

int or_apply_gates_dagger_reversed(int n, double *psi, const or_gate *g, int64_t ng, const double *theta)
{
    int64_t i;
    for (i = ng - 1; i >= 0; i--) {
        int s = apply_gate(n, (cx *)psi, &g[i], theta, 1);
        if (s) return s;
    }
    return OR_OK;
}

/* E = sum_j coeff_j <psi|P_j|psi> (real part; the imaginary part is zero for a Hermitian sum) */
double or_expect(int n, const double *psi, const or_pauli *terms, int64_t nterms)
{
    double e = 0;
    int64_t j;
    for (j = 0; j < nterms; j++) {
        cx v = pauli_braket(n, (const cx *)psi, &terms[j], (const cx *)psi);
        e += terms[j].coeff * v.re;
    }
    return e;
}

/* out = H psi = sum_j coeff_j P_j psi */
void or_apply_hamiltonian(int n, const double *psi_, const or_pauli *terms, int64_t nterms, double *out_)
{
    const cx *psi = (const cx *)psi_;
    cx *out = (cx *)out_;
    uint64_t dim = 1ULL << n;
    int64_t j, k;
    for (k = 0; k < (int64_t)dim; k++) out[k] = cx_make(0, 0);
    for (j = 0; j < nterms; j++) {
        const or_pauli *p = &terms[j];
#pragma omp parallel for schedule(static)
        for (k = 0; k < (int64_t)dim; k++) {
            uint64_t src = (uint64_t)k ^ p->x;
            out[k] = cx_add(out[k], cx_scale(cx_mul(pauli_phase(p, src), psi[src]), p->coeff));
        }
    }
}

/* Adjoint gradient (Jones & Gacon): psi_L = U_L..U_1 |init>, lambda_L = H psi_L,
 * E = Re<psi_L|lambda_L>; for k = L..1: g[param_k] += Im<lambda_k|G_k|psi_k>,
 * then psi_{k-1} = U_k^dagger psi_k and lambda_{k-1} = U_k^dagger lambda_k.
 * Parameterised gates must be uncontrolled RX/RY/RZ (G = X/Y/Z on the target).
 * work: 4 * 2^n doubles provided by the caller. */
int or_adjoint(int n, uint64_t init, const or_gate *g, int64_t ng, const double *theta, int64_t nparams,
               const or_pauli *terms, int64_t nterms, double *energy, double *grad, double *work)
{
    uint64_t dim = 1ULL << n;
    cx *psi = (cx *)work, *lam = (cx *)work + dim;
    int64_t k, p;
    int s;
    for (p = 0; p < nparams; p++) grad[p] = 0;
    memset(psi, 0, sizeof(cx) * dim);
    psi[init] = cx_make(1, 0);
    s = or_apply_gates(n, (double *)psi, g, ng, theta);
    if (s) return s;
    or_apply_hamiltonian(n, (const double *)psi, terms, nterms, (double *)lam);
    {
        double e = 0;
        uint64_t m;
        for (m = 0; m < dim; m++) e += cx_mul(cx_conj(psi[m]), lam[m]).re;
        *energy = e;
    }
    for (k = ng - 1; k >= 0; k--) {
        const or_gate *gk = &g[k];
        if (gk->param >= 0) {
            or_pauli gen;
            cx v;
            if (gk->param >= nparams || gk->nc != 0) return OR_ERR_ARG;
            gen.coeff = 1.0;
            gen.x = gen.z = 0;
            if (gk->kind == OR_RX) gen.x = 1ULL << gk->t[0];
            else if (gk->kind == OR_RY) gen.x = gen.z = 1ULL << gk->t[0];
            else if (gk->kind == OR_RZ) gen.z = 1ULL << gk->t[0];
            else return OR_ERR_ARG;
            v = pauli_braket(n, lam, &gen, psi);
            grad[gk->param] += v.im;
        }
        s = apply_gate(n, psi, gk, theta, 1);
        if (s) return s;
        s = apply_gate(n, lam, gk, theta, 1);
        if (s) return s;
    }
    return OR_OK;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* --------------------------------------------------------------- codec */

#define SVC_MAGIC 0x31435653u

static size_t pad16(size_t x) { return (x + 15) & ~(size_t)15; }

/* exponent k of Delta = 2^k, the largest power of two <= 2*eb */
int or_codec_step_exponent(double eb)
{
    int e;
    double m;
    if (!(eb > 0) || !isfinite(eb)) return 1 << 30;
    m = frexp(2.0 * eb, &e); /* 2 eb = m 2^e, m in [0.5, 1) */
    (void)m;
    return e - 1;
}

static void put32(uint8_t *p, uint32_t v) { p[0] = v & 255; p[1] = (v >> 8) & 255; p[2] = (v >> 16) & 255; p[3] = v >> 24; }
static uint32_t get32(const uint8_t *p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24); }

/* bytes of everything before the payload */
size_t or_codec_meta_bytes(int c)
{
    size_t nb = (size_t)2 << c >> 8;
    return 32 + pad16(nb) + pad16(4 * nb) + pad16(4 * (nb + 1));
}

size_t or_codec_max_bytes(int c)
{
    size_t nb = (size_t)2 << c >> 8;
    return or_codec_meta_bytes(c) + nb * 8 * 32 * 4;
}

static double read_component(int dtype, const void *amps, size_t i, int plane)
{
    if (dtype == 1) return (double)((const float *)amps)[2 * i + plane];
    return ((const double *)amps)[2 * i + plane];
}

/* exponent k of the relative bound's step for a chunk whose largest
 * component magnitude is m: floor(log2(2 eb m)) clamped to [-60, 0] */
int or_codec_relative_exponent(double eb, double m)
{
    int e;
    double f;
    if (!(eb > 0) || !isfinite(eb) || !(m >= 0) || !isfinite(m)) return 1 << 30;
    if (m == 0) return 0;
    f = frexp((2.0 * eb) * m, &e); /* 2 eb m = f 2^e, f in [0.5, 1) */
    (void)f;
    e -= 1;
    return e > 0 ? 0 : e < -60 ? -60 : e;
}

/* largest |re| or |im| of a chunk of 2^c amplitudes */
double or_codec_chunk_max(int dtype, int c, const void *amps)
{
    size_t i, n = (size_t)2 << c;
    double m = 0;
    for (i = 0; i < n; i++) {
        double x = dtype == 1 ? (double)((const float *)amps)[i] : ((const double *)amps)[i];
        if (fabs(x) > m) m = fabs(x);
    }
    return m;
}

static int encode_with_step(int dtype, int c, int k, const void *amps, uint8_t *out, size_t cap, size_t *nbytes);

int or_codec_encode(int dtype, int c, double eb, const void *amps, uint8_t *out, size_t cap, size_t *nbytes)
{
    if ((dtype != 1 && dtype != 2) || c < 8 || c > 30) return OR_ERR_ARG;
    return encode_with_step(dtype, c, or_codec_step_exponent(eb), amps, out, cap, nbytes);
}

int or_codec_encode_relative(int dtype, int c, double eb, const void *amps, uint8_t *out, size_t cap,
                             size_t *nbytes)
{
    if ((dtype != 1 && dtype != 2) || c < 8 || c > 30) return OR_ERR_ARG;
    return encode_with_step(dtype, c, or_codec_relative_exponent(eb, or_codec_chunk_max(dtype, c, amps)), amps, out,
                            cap, nbytes);
}

static int encode_with_step(int dtype, int c, int k, const void *amps, uint8_t *out, size_t cap, size_t *nbytes)
{
    size_t nvals, nb, b, j, meta, w_off, a_off, o_off, p_off, total = 0;
    double qmax, inv;
    int32_t *q;
    uint32_t *z;
    if (k > 0 || k < -60) return OR_ERR_RANGE;
    qmax = dtype == 1 ? 16777215.0 : 1073741823.0;
    inv = ldexp(1.0, -k);
    nvals = (size_t)1 << c;
    nb = 2 * nvals / 256;
    meta = or_codec_meta_bytes(c);
    w_off = 32;
    a_off = w_off + pad16(nb);
    o_off = a_off + pad16(4 * nb);
    p_off = o_off + pad16(4 * (nb + 1));
    if (cap < meta) return OR_ERR_ARG;
    q = (int32_t *)malloc(sizeof(int32_t) * 256);
    z = (uint32_t *)malloc(sizeof(uint32_t) * 256);
    memset(out, 0, meta);
    put32(out + 0, SVC_MAGIC);
    out[4] = 1; out[5] = 0;
    out[6] = (uint8_t)dtype;
    out[7] = (uint8_t)c;
    put32(out + 8, (uint32_t)(int32_t)k);
    put32(out + 12, (uint32_t)nb);
    put32(out + 16 + 0, 0); /* total_words, filled below */
    put32(out + o_off, 0);
    for (b = 0; b < nb; b++) {
        int plane = b < nb / 2 ? 0 : 1;
        size_t first = (b % (nb / 2)) * 256;
        uint32_t maxz = 0;
        int w = 0;
        for (j = 0; j < 256; j++) {
            double x = read_component(dtype, amps, first + j, plane);
            double qd;
            if (!isfinite(x)) { free(q); free(z); return OR_ERR_RANGE; }
            qd = rint(x * inv); /* x * 2^-k is exact; rint rounds half to even */
            if (fabs(qd) > qmax) { free(q); free(z); return OR_ERR_RANGE; }
            q[j] = (int32_t)qd;
        }
        for (j = 0; j < 256; j++) {
            int64_t r = j == 0 ? 0 : (int64_t)q[j] - (int64_t)q[j - 1];
            z[j] = r >= 0 ? (uint32_t)(2 * r) : (uint32_t)(-2 * r - 1);
            if (z[j] > maxz) maxz = z[j];
        }
        while (w < 32 && (maxz >> w) != 0) w++;
        out[w_off + b] = (uint8_t)w;
        put32(out + a_off + 4 * b, (uint32_t)q[0]);
        if (p_off + 4 * (total + 8 * (size_t)w) > cap) { free(q); free(z); return OR_ERR_ARG; }
        /* bit-by-bit packing of z_j into bits [j*w, j*w+w) */
        memset(out + p_off + 4 * total, 0, 4 * 8 * (size_t)w);
        for (j = 0; j < 256; j++) {
            int bit;
            for (bit = 0; bit < w; bit++) {
                if ((z[j] >> bit) & 1) {
                    size_t pos = j * (size_t)w + (size_t)bit;
                    out[p_off + 4 * total + pos / 8] |= (uint8_t)(1u << (pos % 8));
                }
            }
        }
        total += 8 * (size_t)w;
        put32(out + o_off + 4 * (b + 1), (uint32_t)total);
    }
    put32(out + 16, (uint32_t)total);
    *nbytes = p_off + 4 * total;
    free(q);
    free(z);
    return OR_OK;
}

int or_codec_decode(int dtype, int c, const uint8_t *in, size_t nbytes, void *amps)
{
    size_t nvals, nb, b, j, w_off, a_off, o_off, p_off, total;
    int k;
    double delta;
    if ((dtype != 1 && dtype != 2) || c < 8 || c > 30) return OR_ERR_ARG;
    if (nbytes < or_codec_meta_bytes(c)) return OR_ERR_CORRUPT;
    if (get32(in) != SVC_MAGIC || in[4] != 1 || in[5] != 0 || in[6] != dtype || in[7] != c) return OR_ERR_CORRUPT;
    k = (int32_t)get32(in + 8);
    if (k > 0 || k < -60) return OR_ERR_CORRUPT;
    delta = ldexp(1.0, k);
    nvals = (size_t)1 << c;
    nb = 2 * nvals / 256;
    if (get32(in + 12) != nb) return OR_ERR_CORRUPT;
    total = get32(in + 16);
    w_off = 32;
    a_off = w_off + pad16(nb);
    o_off = a_off + pad16(4 * nb);
    p_off = o_off + pad16(4 * (nb + 1));
    if (p_off + 4 * total > nbytes) return OR_ERR_CORRUPT;
    if (get32(in + o_off) != 0 || get32(in + o_off + 4 * nb) != total) return OR_ERR_CORRUPT;
    for (b = 0; b < nb; b++) {
        int plane = b < nb / 2 ? 0 : 1;
        size_t first = (b % (nb / 2)) * 256;
        int w = in[w_off + b];
        uint32_t off = get32(in + o_off + 4 * b);
        int32_t qv;
        if (w > 32 || get32(in + o_off + 4 * (b + 1)) - off != 8u * (uint32_t)w) return OR_ERR_CORRUPT;
        qv = (int32_t)get32(in + a_off + 4 * b);
        for (j = 0; j < 256; j++) {
            uint32_t zj = 0;
            int64_t r;
            double x;
            int bit;
            for (bit = 0; bit < w; bit++) {
                size_t pos = j * (size_t)w + (size_t)bit;
                if ((in[p_off + 4 * (size_t)off + pos / 8] >> (pos % 8)) & 1) zj |= 1u << bit;
            }
            r = (zj & 1) ? -(int64_t)((zj >> 1) + 1) : (int64_t)(zj >> 1);
            if (j > 0) qv = (int32_t)(uint32_t)((int64_t)qv + r); /* wrap-around add, as int32 */
            x = (double)qv * delta; /* exact */
            if (dtype == 1) ((float *)amps)[2 * (first + j) + plane] = (float)x;
            else ((double *)amps)[2 * (first + j) + plane] = x;
        }
    }
    return OR_OK;
}
