/*
 * CPU oracle for the GPU-aware OpenSHMEM operations on a symmetric heap.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this file's library; the product path never does.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * Model (paper, Sec. 2.1 and Fig. 1): a symmetric heap of npes partitions of H bytes
 * each.  The byte at symmetric offset o on PE p is heap[p*H + o].  Every operation is
 * applied one at a time, by its definition, in plain sequential C: no blocking, no
 * fusion, no reordering.  Float arithmetic is IEEE binary32/binary64 with round to
 * nearest even; build with -O2 -ffp-contract=off and without -ffast-math.
 *
 * Operation meanings are inherited unchanged from OpenSHMEM 1.6 (paper, Sec. 6.3:
 * symmetric allocation, team collectivity, fence/quiet).  The readings used where the
 * paper is silent are listed beside each function.
 *
 * Parity status: every function below is pinned by a CPU test against the
 * mathematics (closed forms, brute force, hand-computed fixtures, invariants); none is
 * "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_RANGE (-1)
#define OR_ERR_ARG (-2)
#define OR_ERR_WAIT (-3)
#define OR_ERR_NOMEM (-4)

/* op kinds of a scripted operation record (64 bytes, little endian) */
enum {
    K_PUT = 1, K_GET = 2, K_PUT_NBI = 3, K_GET_NBI = 4,
    K_FADD = 5, K_CSWAP = 6, K_FXOR = 7,
    K_PUT_SIGNAL = 8, K_WAIT_UNTIL = 9,
    K_BARRIER_ALL = 10, K_QUIET = 11, K_FENCE = 12,
    K_BCAST = 13, K_FCOLLECT = 14, K_ALLTOALL = 15, K_REDUCE = 16, K_TEAM_SYNC = 17
};
enum { T_I32 = 0, T_I64 = 1, T_F32 = 2, T_U64 = 3 };
enum { R_SUM = 0, R_MAX = 1, R_MIN = 2 };
enum { S_SET = 0, S_ADD = 1 };
enum { C_EQ = 0, C_NE, C_GT, C_GE, C_LT, C_LE };
enum { F_BF16 = 0, F_E4M3 = 1 };

typedef struct {
    uint32_t kind;
    uint8_t dtype;
    uint8_t sub;
    uint16_t team;
    int32_t pe;
    int32_t issuer;
    uint64_t dst;
    uint64_t src;
    uint64_t n;
    int64_t operand;
    int64_t cond;
    uint64_t aux;
} or_op;

typedef struct {
    uint8_t *base;
    int npes;
    uint64_t H;
} heap_t;

static int in_range(const heap_t *h, int pe, uint64_t off, uint64_t n) {
    return pe >= 0 && pe < h->npes && off <= h->H && n <= h->H - off;
}

static uint8_t *at(const heap_t *h, int pe, uint64_t off) {
    return h->base + (uint64_t)pe * h->H + off;
}

/* team member r (0-based team rank) -> PE, for a strided team (OpenSHMEM 1.6 teams) */
static int member(int start, int stride, int r) { return start + r * stride; }

/* ------------------------------------------------------------------ RMA (Sec. 2.1) */
/* put: dst on dst_pe <- src on src_pe, nbytes.  get is the same copy with the roles of
 * local and remote swapped; _nbi forms have the same final state once quiet returns
 * (Sec. 6.3: non-blocking operations complete at quiet). */
int or_copy(uint8_t *base, int npes, uint64_t H, int dst_pe, uint64_t dst, int src_pe,
            uint64_t src, uint64_t nbytes) {
    heap_t h = {base, npes, H};
    if (!in_range(&h, dst_pe, dst, nbytes) || !in_range(&h, src_pe, src, nbytes))
        return OR_ERR_RANGE;
    uint8_t *tmp = (uint8_t *)malloc(nbytes ? nbytes : 1);
    if (!tmp) return OR_ERR_NOMEM;
    for (uint64_t i = 0; i < nbytes; i++) tmp[i] = at(&h, src_pe, src)[i];
    for (uint64_t i = 0; i < nbytes; i++) at(&h, dst_pe, dst)[i] = tmp[i];
    free(tmp);
    return OR_OK;
}

/* ------------------------------------------------------------------ AMO (Sec. 2.1) */
/* fetch_add returns the old value and stores old + v (two's complement wraparound);
 * compare_swap returns the old value and stores v iff old == cond; fetch_xor returns
 * the old value and stores old ^ v.  Atomicity only: ordering needs fence/quiet
 * (Sec. 6.3). */
int or_amo64(uint8_t *base, int npes, uint64_t H, int kind, int pe, uint64_t off,
             int64_t v, int64_t cond, int64_t *fetched) {
    heap_t h = {base, npes, H};
    if (!in_range(&h, pe, off, 8) || (off & 7)) return OR_ERR_RANGE;
    int64_t old;
    memcpy(&old, at(&h, pe, off), 8);
    uint64_t nw;
    if (kind == K_FADD) nw = (uint64_t)old + (uint64_t)v;
    else if (kind == K_CSWAP) nw = (old == cond) ? (uint64_t)v : (uint64_t)old;
    else if (kind == K_FXOR) nw = (uint64_t)old ^ (uint64_t)v;
    else return OR_ERR_ARG;
    memcpy(at(&h, pe, off), &nw, 8);
    if (fetched) *fetched = old;
    return OR_OK;
}

int or_amo32(uint8_t *base, int npes, uint64_t H, int kind, int pe, uint64_t off,
             int32_t v, int32_t cond, int32_t *fetched) {
    heap_t h = {base, npes, H};
    if (!in_range(&h, pe, off, 4) || (off & 3)) return OR_ERR_RANGE;
    int32_t old;
    memcpy(&old, at(&h, pe, off), 4);
    uint32_t nw;
    if (kind == K_FADD) nw = (uint32_t)old + (uint32_t)v;
    else if (kind == K_CSWAP) nw = (old == cond) ? (uint32_t)v : (uint32_t)old;
    else if (kind == K_FXOR) nw = (uint32_t)old ^ (uint32_t)v;
    else return OR_ERR_ARG;
    memcpy(at(&h, pe, off), &nw, 4);
    if (fetched) *fetched = old;
    return OR_OK;
}

/* ------------------------------------------------------- signals (Sec. 7, put-signal) */
/* put_signal: the data put, then the signal word (uint64, in the symmetric heap) is set
 * to v (SET) or incremented by v with wraparound (ADD). */
int or_put_signal(uint8_t *base, int npes, uint64_t H, int dst_pe, uint64_t dst, int src_pe,
                  uint64_t src, uint64_t nbytes, uint64_t sig_off, int sig_op, uint64_t v) {
    heap_t h = {base, npes, H};
    if (!in_range(&h, dst_pe, sig_off, 8) || (sig_off & 7)) return OR_ERR_RANGE;
    int rc = or_copy(base, npes, H, dst_pe, dst, src_pe, src, nbytes);
    if (rc) return rc;
    uint64_t s;
    memcpy(&s, at(&h, dst_pe, sig_off), 8);
    if (sig_op == S_SET) s = v;
    else if (sig_op == S_ADD) s = s + v;
    else return OR_ERR_ARG;
    memcpy(at(&h, dst_pe, sig_off), &s, 8);
    return OR_OK;
}

/* wait_until / test on a uint64 signal word: 1 if "sig cmp v" holds, 0 if not. */
int or_signal_test(uint8_t *base, int npes, uint64_t H, int pe, uint64_t off, int cmp,
                   uint64_t v) {
    heap_t h = {base, npes, H};
    if (!in_range(&h, pe, off, 8) || (off & 7)) return OR_ERR_RANGE;
    uint64_t s;
    memcpy(&s, at(&h, pe, off), 8);
    switch (cmp) {
    case C_EQ: return s == v;
    case C_NE: return s != v;
    case C_GT: return s > v;
    case C_GE: return s >= v;
    case C_LT: return s < v;
    case C_LE: return s <= v;
    default: return OR_ERR_ARG;
    }
}

/* ------------------------------------------------------ collectives (OpenSHMEM 1.6) */
static int team_ok(const heap_t *h, int start, int stride, int size) {
    if (size < 1 || start < 0 || stride < 1) return 0;
    return member(start, stride, size - 1) < h->npes;
}

/* broadcast: every member's dst (the root's included) receives the root's src;
 * root is a team rank. */
int or_broadcast(uint8_t *base, int npes, uint64_t H, int start, int stride, int size,
                 uint64_t dst, uint64_t src, uint64_t nbytes, int root) {
    heap_t h = {base, npes, H};
    if (!team_ok(&h, start, stride, size) || root < 0 || root >= size) return OR_ERR_ARG;
    if (!in_range(&h, 0, dst, nbytes) || !in_range(&h, 0, src, nbytes)) return OR_ERR_RANGE;
    uint8_t *tmp = (uint8_t *)malloc(nbytes ? nbytes : 1);
    if (!tmp) return OR_ERR_NOMEM;
    memcpy(tmp, at(&h, member(start, stride, root), src), nbytes);
    for (int r = 0; r < size; r++) memcpy(at(&h, member(start, stride, r), dst), tmp, nbytes);
    free(tmp);
    return OR_OK;
}

/* fcollect: member p's dst holds, at byte offset r*nbytes, member r's src (team-rank
 * order), for every member p. */
int or_fcollect(uint8_t *base, int npes, uint64_t H, int start, int stride, int size,
                uint64_t dst, uint64_t src, uint64_t nbytes) {
    heap_t h = {base, npes, H};
    if (!team_ok(&h, start, stride, size)) return OR_ERR_ARG;
    uint64_t total = nbytes * (uint64_t)size;
    if (!in_range(&h, 0, dst, total) || !in_range(&h, 0, src, nbytes)) return OR_ERR_RANGE;
    uint8_t *tmp = (uint8_t *)malloc(total ? total : 1);
    if (!tmp) return OR_ERR_NOMEM;
    for (int r = 0; r < size; r++)
        memcpy(tmp + (uint64_t)r * nbytes, at(&h, member(start, stride, r), src), nbytes);
    for (int p = 0; p < size; p++) memcpy(at(&h, member(start, stride, p), dst), tmp, total);
    free(tmp);
    return OR_OK;
}

/* alltoall: member j's dst block i <- member i's src block j (blocks of m bytes). */
int or_alltoall(uint8_t *base, int npes, uint64_t H, int start, int stride, int size,
                uint64_t dst, uint64_t src, uint64_t m) {
    heap_t h = {base, npes, H};
    if (!team_ok(&h, start, stride, size)) return OR_ERR_ARG;
    uint64_t total = m * (uint64_t)size;
    if (!in_range(&h, 0, dst, total) || !in_range(&h, 0, src, total)) return OR_ERR_RANGE;
    uint64_t all = total * (uint64_t)size;
    uint8_t *tmp = (uint8_t *)malloc(all ? all : 1);
    if (!tmp) return OR_ERR_NOMEM;
    /* tmp[j][i] = member i's src block j */
    for (int i = 0; i < size; i++)
        for (int j = 0; j < size; j++)
            memcpy(tmp + ((uint64_t)j * size + i) * m,
                   at(&h, member(start, stride, i), src + (uint64_t)j * m), m);
    for (int j = 0; j < size; j++)
        memcpy(at(&h, member(start, stride, j), dst), tmp + (uint64_t)j * size * m, total);
    free(tmp);
    return OR_OK;
}

/* Fixed float reduction order: the rank-pairwise tree.  Level 0 holds the members'
 * values in team-rank order; each level replaces the pairs (2i, 2i+1) by their binary32
 * sum and carries an odd last element up unchanged, until one value is left. */
float or_tree_sum_f32(float *v, int count) {
    int m = count;
    if (m <= 0) return 0.0f;
    while (m > 1) {
        int k = 0;
        for (int i = 0; i + 1 < m; i += 2) {
            volatile float s = v[i] + v[i + 1];
            v[k++] = s;
        }
        if (m & 1) v[k++] = v[m - 1];
        m = k;
    }
    return v[0];
}

/* reduce with all-reduce semantics: every member's dst[k] = op over members of
 * src[k].  Integer sums wrap (two's complement); float sum uses the pairwise tree;
 * max/min are exact.  dst == src (in place) is allowed: all inputs are read first. */
int or_reduce(uint8_t *base, int npes, uint64_t H, int start, int stride, int size,
              uint64_t dst, uint64_t src, uint64_t nelems, int dtype, int op) {
    heap_t h = {base, npes, H};
    if (!team_ok(&h, start, stride, size)) return OR_ERR_ARG;
    uint64_t es = (dtype == T_I32 || dtype == T_F32) ? 4 : 8;
    if (dtype != T_I32 && dtype != T_I64 && dtype != T_F32) return OR_ERR_ARG;
    if (op != R_SUM && op != R_MAX && op != R_MIN) return OR_ERR_ARG;
    if (!in_range(&h, 0, dst, nelems * es) || !in_range(&h, 0, src, nelems * es))
        return OR_ERR_RANGE;
    uint8_t *in = (uint8_t *)malloc(nelems * es * (uint64_t)size + 1);
    uint8_t *out = (uint8_t *)malloc(nelems * es + 1);
    float *col = (float *)malloc(sizeof(float) * (uint64_t)size);
    if (!in || !out || !col) { free(in); free(out); free(col); return OR_ERR_NOMEM; }
    for (int r = 0; r < size; r++)
        memcpy(in + (uint64_t)r * nelems * es, at(&h, member(start, stride, r), src), nelems * es);
    for (uint64_t k = 0; k < nelems; k++) {
        if (dtype == T_I64) {
            int64_t acc;
            memcpy(&acc, in + k * 8, 8);
            for (int r = 1; r < size; r++) {
                int64_t x;
                memcpy(&x, in + ((uint64_t)r * nelems + k) * 8, 8);
                if (op == R_SUM) acc = (int64_t)((uint64_t)acc + (uint64_t)x);
                else if (op == R_MAX) acc = x > acc ? x : acc;
                else acc = x < acc ? x : acc;
            }
            memcpy(out + k * 8, &acc, 8);
        } else if (dtype == T_I32) {
            int32_t acc;
            memcpy(&acc, in + k * 4, 4);
            for (int r = 1; r < size; r++) {
                int32_t x;
                memcpy(&x, in + ((uint64_t)r * nelems + k) * 4, 4);
                if (op == R_SUM) acc = (int32_t)((uint32_t)acc + (uint32_t)x);
                else if (op == R_MAX) acc = x > acc ? x : acc;
                else acc = x < acc ? x : acc;
            }
            memcpy(out + k * 4, &acc, 4);
        } else {
            for (int r = 0; r < size; r++) memcpy(&col[r], in + ((uint64_t)r * nelems + k) * 4, 4);
            float acc;
            if (op == R_SUM) {
                acc = or_tree_sum_f32(col, size);
            } else {
                acc = col[0];
                for (int r = 1; r < size; r++) {
                    if (op == R_MAX) acc = col[r] > acc ? col[r] : acc;
                    else acc = col[r] < acc ? col[r] : acc;
                }
            }
            memcpy(out + k * 4, &acc, 4);
        }
    }
    for (int r = 0; r < size; r++) memcpy(at(&h, member(start, stride, r), dst), out, nelems * es);
    free(in);
    free(out);
    free(col);
    return OR_OK;
}

/* binary64 reference of a float sum reduce, for the error gate: y64[k] = sum over
 * members in rank order of (double)x_r[k], and abs64[k] = sum of |x_r[k]|. */
int or_reduce_f32_ref64(const uint8_t *base, int npes, uint64_t H, int start, int stride,
                        int size, uint64_t src, uint64_t nelems, double *y64, double *abs64) {
    heap_t h = {(uint8_t *)base, npes, H};
    if (!team_ok(&h, start, stride, size)) return OR_ERR_ARG;
    if (!in_range(&h, 0, src, nelems * 4)) return OR_ERR_RANGE;
    for (uint64_t k = 0; k < nelems; k++) {
        double s = 0.0, a = 0.0;
        for (int r = 0; r < size; r++) {
            float x;
            memcpy(&x, at(&h, member(start, stride, r), src) + k * 4, 4);
            s += (double)x;
            a += fabs((double)x);
        }
        y64[k] = s;
        abs64[k] = a;
    }
    return OR_OK;
}

/* ------------------------------------------------------------ quantised payloads */
/* bfloat16: the top 16 bits of a binary32 (1 sign, 8 exponent, 7 mantissa bits).
 * Decoding appends 16 zero bits. */
float or_bf16_decode(uint16_t q) {
    uint32_t b = (uint32_t)q << 16;
    float f;
    memcpy(&f, &b, 4);
    return f;
}

/* Encoding by definition: of the two bfloat16 values that bracket x (truncation toward
 * zero and the next one away from zero), take the nearer; on a tie take the one whose
 * last mantissa bit is 0 (round to nearest even).  Finite inputs only. */
uint16_t or_bf16_encode(float x) {
    uint32_t b;
    memcpy(&b, &x, 4);
    uint16_t lo = (uint16_t)(b >> 16);          /* toward zero */
    if ((b & 0xFFFFu) == 0) return lo;
    uint16_t hi = (uint16_t)(lo + 1);           /* away from zero (same sign) */
    double dx = fabs((double)x);
    double dlo = fabs((double)or_bf16_decode(lo));
    double dhi = fabs((double)or_bf16_decode(hi));
    double elo = dx - dlo, ehi = dhi - dx;
    if (elo < ehi) return lo;
    if (ehi < elo) return hi;
    return (lo & 1) ? hi : lo;
}

/* OCP FP8 E4M3 ("E4M3FN"): 1 sign, 4 exponent bits (bias 7), 3 mantissa bits, no
 * infinities, S.1111.111 is NaN, largest finite 448 = 1.75 * 2^8, smallest normal
 * 2^-6, subnormals m/8 * 2^-6 down to 2^-9. */
double or_e4m3_decode(uint8_t q) {
    int s = q >> 7, e = (q >> 3) & 15, m = q & 7;
    double v;
    if (e == 15 && m == 7) return NAN;
    if (e == 0) v = ldexp((double)m / 8.0, -6);
    else v = ldexp(1.0 + (double)m / 8.0, e - 7);
    return s ? -v : v;
}

/* Encoding by definition: magnitude -> the nearest of the 127 non-negative finite
 * codes (0x00..0x7E) by exhaustive search; ties go to the even code (mantissa bit 0);
 * magnitudes above 448 saturate to 448; the sign bit is copied from x. */
uint8_t or_e4m3_encode(float x) {
    double a = fabs((double)x);
    uint8_t best = 0;
    if (a >= 448.0) {
        best = 0x7E;
    } else {
        double bd = INFINITY;
        for (int c = 0; c <= 0x7E; c++) {
            double d = fabs(or_e4m3_decode((uint8_t)c) - a);
            if (d < bd || (d == bd && (c & 1) == 0)) {
                bd = d;
                best = (uint8_t)c;
            }
        }
    }
    return signbit(x) ? (uint8_t)(best | 0x80) : best;
}

/* Block quantisation of one PE's n floats in blocks of 128 (last block may be short):
 * amax = max|x|, s = amax / R (binary32 divide; R = 448 for e4m3, 1 for bf16; s = 1
 * when amax = 0), q = enc(x / s) (binary32 divide, then RNE with saturation). */
int or_quantize(const float *x, uint64_t n, int fmt, void *q, float *scales) {
    if (fmt != F_BF16 && fmt != F_E4M3) return OR_ERR_ARG;
    const float R = (fmt == F_E4M3) ? 448.0f : 1.0f;
    for (uint64_t b = 0; b * 128 < n; b++) {
        uint64_t lo = b * 128, hi = lo + 128 < n ? lo + 128 : n;
        float amax = 0.0f;
        for (uint64_t i = lo; i < hi; i++) {
            float a = fabsf(x[i]);
            if (a > amax) amax = a;
        }
        volatile float s = (amax == 0.0f) ? 1.0f : amax / R;
        scales[b] = s;
        for (uint64_t i = lo; i < hi; i++) {
            volatile float y = x[i] / s;
            if (fmt == F_E4M3) ((uint8_t *)q)[i] = or_e4m3_encode(y);
            else ((uint16_t *)q)[i] = or_bf16_encode(y);
        }
    }
    return OR_OK;
}

/* Dequantised value of element i: float(q_i) * s_(i/128), one binary32 multiply. */
static float deq(const void *q, const float *scales, uint64_t i, int fmt) {
    float v = (fmt == F_E4M3) ? (float)or_e4m3_decode(((const uint8_t *)q)[i])
                              : or_bf16_decode(((const uint16_t *)q)[i]);
    volatile float r = v * scales[i / 128];
    return r;
}

/* Neumaier's compensated summation in binary32 over the given order:
 * t = sum + x; c += (sum - t) + x if |sum| >= |x| else (x - t) + sum; sum = t;
 * the result is sum + c. */
float or_neumaier_f32(const float *x, int count) {
    volatile float sum = 0.0f, c = 0.0f;
    for (int i = 0; i < count; i++) {
        volatile float t = sum + x[i];
        if (fabsf(sum) >= fabsf(x[i])) {
            volatile float d = sum - t;
            c = c + (d + x[i]);
        } else {
            volatile float d = x[i] - t;
            c = c + (d + sum);
        }
        sum = t;
    }
    volatile float y = sum + c;
    return y;
}

/* Quantised sum reduce (all-reduce): member p's float dst[k] = Neumaier sum, in team
 * rank order, of the dequantised payloads of every member.  Payload q (n codes) and
 * scales (ceil(n/128) floats) are symmetric objects at offsets q_off and s_off. */
int or_qsum_reduce(uint8_t *base, int npes, uint64_t H, int start, int stride, int size,
                   uint64_t dst, uint64_t q_off, uint64_t s_off, int fmt, uint64_t n) {
    heap_t h = {base, npes, H};
    if (!team_ok(&h, start, stride, size)) return OR_ERR_ARG;
    uint64_t qs = (fmt == F_E4M3) ? 1 : 2, nb = (n + 127) / 128;
    if (!in_range(&h, 0, dst, n * 4) || !in_range(&h, 0, q_off, n * qs) ||
        !in_range(&h, 0, s_off, nb * 4))
        return OR_ERR_RANGE;
    float *out = (float *)malloc(n * 4 + 4);
    float *col = (float *)malloc(sizeof(float) * (uint64_t)size);
    if (!out || !col) { free(out); free(col); return OR_ERR_NOMEM; }
    for (uint64_t k = 0; k < n; k++) {
        for (int r = 0; r < size; r++) {
            int p = member(start, stride, r);
            col[r] = deq(at(&h, p, q_off), (const float *)at(&h, p, s_off), k, fmt);
        }
        out[k] = or_neumaier_f32(col, size);
    }
    for (int r = 0; r < size; r++) memcpy(at(&h, member(start, stride, r), dst), out, n * 4);
    free(out);
    free(col);
    return OR_OK;
}

/* binary64 sum of the dequantised payloads (accumulation-error reference). */
int or_qsum_ref64(const uint8_t *base, int npes, uint64_t H, int start, int stride, int size,
                  uint64_t q_off, uint64_t s_off, int fmt, uint64_t n, double *y64,
                  double *abs64) {
    heap_t h = {(uint8_t *)base, npes, H};
    if (!team_ok(&h, start, stride, size)) return OR_ERR_ARG;
    for (uint64_t k = 0; k < n; k++) {
        double s = 0.0, a = 0.0;
        for (int r = 0; r < size; r++) {
            int p = member(start, stride, r);
            double v = (double)deq(at(&h, p, q_off), (const float *)at(&h, p, s_off), k, fmt);
            s += v;
            a += fabs(v);
        }
        y64[k] = s;
        abs64[k] = a;
    }
    return OR_OK;
}

/* --------------------------------------------------------------- script execution */
/* Runs a scripted operation list in script order (the sequential reference for both
 * the launch-per-op path and the device-initiated interpreter).  teams[3*t..3*t+2] =
 * (start, stride, size) of team t.  fetched[i] receives the old value of AMO op i.
 * Barriers, fences and quiets have no effect on data.  A wait_until whose condition
 * does not hold when reached is an error (a sequential program would never return). */
int or_run_script(uint8_t *base, int npes, uint64_t H, const or_op *ops, int64_t nops,
                  const int32_t *teams, int nteams, int64_t *fetched, int64_t *failed_op) {
    for (int64_t i = 0; i < nops; i++) {
        const or_op *o = &ops[i];
        int rc = OR_OK;
        int ts = 0, tstr = 1, tsz = npes;
        if (o->team < nteams) {
            ts = teams[3 * o->team];
            tstr = teams[3 * o->team + 1];
            tsz = teams[3 * o->team + 2];
        } else if (o->kind >= K_BCAST) {
            rc = OR_ERR_ARG;
        }
        if (rc == OR_OK) switch (o->kind) {
        case K_PUT: case K_PUT_NBI:
            rc = or_copy(base, npes, H, o->pe, o->dst, o->issuer, o->src, o->n);
            break;
        case K_GET: case K_GET_NBI:
            rc = or_copy(base, npes, H, o->issuer, o->dst, o->pe, o->src, o->n);
            break;
        case K_FADD: case K_CSWAP: case K_FXOR:
            if (o->dtype == T_I64) {
                rc = or_amo64(base, npes, H, (int)o->kind, o->pe, o->dst, o->operand, o->cond,
                              &fetched[i]);
            } else if (o->dtype == T_I32) {
                int32_t f = 0;
                rc = or_amo32(base, npes, H, (int)o->kind, o->pe, o->dst, (int32_t)o->operand,
                              (int32_t)o->cond, &f);
                fetched[i] = f;
            } else {
                rc = OR_ERR_ARG;
            }
            break;
        case K_PUT_SIGNAL:
            rc = or_put_signal(base, npes, H, o->pe, o->dst, o->issuer, o->src, o->n, o->aux,
                               o->sub, (uint64_t)o->operand);
            break;
        case K_WAIT_UNTIL: {
            int t = or_signal_test(base, npes, H, o->issuer, o->dst, o->sub, (uint64_t)o->operand);
            rc = t < 0 ? t : (t ? OR_OK : OR_ERR_WAIT);
            break;
        }
        case K_BARRIER_ALL: case K_QUIET: case K_FENCE: case K_TEAM_SYNC:
            break;
        case K_BCAST:
            rc = or_broadcast(base, npes, H, ts, tstr, tsz, o->dst, o->src, o->n, o->pe);
            break;
        case K_FCOLLECT:
            rc = or_fcollect(base, npes, H, ts, tstr, tsz, o->dst, o->src, o->n);
            break;
        case K_ALLTOALL:
            rc = or_alltoall(base, npes, H, ts, tstr, tsz, o->dst, o->src, o->n);
            break;
        case K_REDUCE:
            rc = or_reduce(base, npes, H, ts, tstr, tsz, o->dst, o->src, o->n, o->dtype, o->sub);
            break;
        default:
            rc = OR_ERR_ARG;
        }
        if (rc != OR_OK) {
            if (failed_op) *failed_op = i;
            return rc;
        }
    }
    return OR_OK;
}

/* -------------------------------------------------------------- AMO stress stream */
/* splitmix64 (Steele, Lea, Flood, OOPSLA 2014): state += 0x9E3779B97F4A7C15, then the
 * output mix.  cb64(seed, i) is the first output of the stream seeded with seed ^ i. */
uint64_t or_cb64(uint64_t seed, uint64_t i) {
    uint64_t z = (seed ^ i) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Sequential application of a packed AMO stream to an int64 table.  Op i: word =
 * bits 0..26, code = bits 27..28 (0 fetch_add, 1 compare_swap, 2 fetch_xor).  Its
 * operand r = cb64(op_seed, first_op + i); fetch_add adds (r mod 2^20) + 1;
 * compare_swap's condition is the word's initial value cb64(table_seed, word) and its
 * new value r; fetch_xor xors r (1 if r is 0).  fetched may be NULL. */
int or_amo_stream(int64_t *table, uint64_t nwords, const uint32_t *ops, uint64_t count,
                  uint64_t first_op, uint64_t op_seed, uint64_t table_seed, int64_t *fetched) {
    for (uint64_t i = 0; i < count; i++) {
        uint64_t w = ops[i] & ((1u << 27) - 1);
        unsigned code = (ops[i] >> 27) & 3;
        if (w >= nwords) return OR_ERR_RANGE;
        uint64_t r = or_cb64(op_seed, first_op + i);
        int64_t old = table[w];
        uint64_t nw;
        if (code == 0) nw = (uint64_t)old + (r % (1u << 20)) + 1;
        else if (code == 1) nw = ((uint64_t)old == or_cb64(table_seed, w)) ? r : (uint64_t)old;
        else if (code == 2) nw = (uint64_t)old ^ (r ? r : 1);
        else return OR_ERR_ARG;
        table[w] = (int64_t)nw;
        if (fetched) fetched[i] = old;
    }
    return OR_OK;
}

/* ------------------------------------------------------- serialisation checker */
/* Concurrent AMOs on one word are correct iff some order of them, replayed from the
 * word's starting value w0, reproduces every fetched value (and the final value, when
 * given).  Depth-first search: at each value, first place every unplaced op that does
 * not change the word at that value and fetched it (placing it now is always as good as
 * later), then branch over the unplaced ops that change it and fetched it.
 * Ops: kind (K_FADD/K_CSWAP/K_FXOR), operand, cond, fetched; one group per word. */
typedef struct { int64_t fetched; int64_t idx; } fe_t;

static int fe_cmp(const void *a, const void *b) {
    const fe_t *x = (const fe_t *)a, *y = (const fe_t *)b;
    if (x->fetched != y->fetched) return x->fetched < y->fetched ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int64_t apply1(int kind, int64_t cur, int64_t v, int64_t c) {
    if (kind == K_FADD) return (int64_t)((uint64_t)cur + (uint64_t)v);
    if (kind == K_CSWAP) return cur == c ? v : cur;
    return (int64_t)((uint64_t)cur ^ (uint64_t)v);
}

/* returns 1 valid, 0 invalid, -1 search budget exhausted */
static int check_group(int64_t n, const int32_t *kind, const int64_t *operand,
                       const int64_t *cond, const fe_t *sorted, int64_t w0, int has_final,
                       int64_t final, int64_t budget) {
    uint8_t *placed = (uint8_t *)calloc((size_t)n + 1, 1);
    int64_t *trail = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    /* choice frames: value before, position of the chosen candidate, trail length */
    int64_t *fr_val = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int64_t *fr_pos = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int64_t *fr_len = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!placed || !trail || !fr_val || !fr_pos || !fr_len) {
        free(placed); free(trail); free(fr_val); free(fr_pos); free(fr_len);
        return -1;
    }
    int64_t ntrail = 0, nfr = 0, cur = w0, start_pos = 0;
    int result = 0;
    for (;;) {
        if (--budget < 0) { result = -1; break; }
        /* bucket of ops whose fetched value equals cur */
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (sorted[mid].fetched < cur) lo = mid + 1; else hi = mid;
        }
        int64_t b0 = lo, b1 = lo;
        while (b1 < n && sorted[b1].fetched == cur) b1++;
        /* forced placements: ops that leave the word unchanged at cur */
        for (int64_t p = b0; p < b1; p++) {
            int64_t j = sorted[p].idx;
            if (!placed[j] && apply1(kind[j], cur, operand[j], cond[j]) == cur) {
                placed[j] = 1;
                trail[ntrail++] = j;
            }
        }
        if (ntrail == n) {
            if (!has_final || cur == final) { result = 1; break; }
        } else {
            int64_t p = b0 > start_pos ? b0 : start_pos;
            for (; p < b1; p++) {
                int64_t j = sorted[p].idx;
                if (!placed[j]) break;
            }
            if (p < b1) {
                int64_t j = sorted[p].idx;
                fr_val[nfr] = cur; fr_pos[nfr] = p; fr_len[nfr] = ntrail; nfr++;
                placed[j] = 1;
                trail[ntrail++] = j;
                cur = apply1(kind[j], cur, operand[j], cond[j]);
                start_pos = 0;
                continue;
            }
        }
        /* backtrack */
        if (nfr == 0) { result = 0; break; }
        nfr--;
        while (ntrail > fr_len[nfr]) placed[trail[--ntrail]] = 0;
        cur = fr_val[nfr];
        start_pos = fr_pos[nfr] + 1;
    }
    free(placed); free(trail); free(fr_val); free(fr_pos); free(fr_len);
    return result;
}

/* Checks every word group.  group[i] identifies op i's word (ops of one group need not
 * be adjacent); w0[i] / final[i] give that word's starting / final value (the same for
 * every op of a group).  Returns the number of invalid groups, or -1 if the search
 * budget ran out on some group (inconclusive); *bad_group receives one failing group. */
int64_t or_check_serialisation(int64_t n, const int64_t *group, const int32_t *kind,
                               const int64_t *operand, const int64_t *cond,
                               const int64_t *fetched, const int64_t *w0, const int64_t *final,
                               int has_final, int64_t budget_per_group, int64_t *bad_group) {
    fe_t *ord = (fe_t *)malloc(sizeof(fe_t) * ((size_t)n + 1));
    if (!ord) return -1;
    for (int64_t i = 0; i < n; i++) { ord[i].fetched = group[i]; ord[i].idx = i; }
    qsort(ord, (size_t)n, sizeof(fe_t), fe_cmp); /* by group, then index */
    int32_t *gk = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int64_t *gv = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int64_t *gc = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    fe_t *gs = (fe_t *)malloc(sizeof(fe_t) * ((size_t)n + 1));
    int64_t bad = 0;
    int inconclusive = 0;
    for (int64_t a = 0; a < n;) {
        int64_t b = a;
        while (b < n && ord[b].fetched == ord[a].fetched) b++;
        int64_t m = b - a;
        for (int64_t t = 0; t < m; t++) {
            int64_t i = ord[a + t].idx;
            gk[t] = kind[i];
            gv[t] = operand[i];
            gc[t] = cond[i];
            gs[t].fetched = fetched[i];
            gs[t].idx = t;
        }
        qsort(gs, (size_t)m, sizeof(fe_t), fe_cmp);
        int64_t i0 = ord[a].idx;
        int r = check_group(m, gk, gv, gc, gs, w0[i0], has_final, has_final ? final[i0] : 0,
                            budget_per_group);
        if (r == 0) {
            bad++;
            if (bad_group) *bad_group = group[i0];
        } else if (r < 0) {
            inconclusive = 1;
            if (bad_group) *bad_group = group[i0];
        }
        a = b;
    }
    free(ord); free(gk); free(gv); free(gc); free(gs);
    return inconclusive && bad == 0 ? -1 : bad;
}
