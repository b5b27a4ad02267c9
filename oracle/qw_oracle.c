/*
 * qw_oracle.c -- plain, slow, obviously-correct CPU reference for the
 * workload-reuse hot path.  TEST INFRASTRUCTURE ONLY: nothing in the product
 * library links, includes or calls this file; only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.
 *
 * What it computes (and why that is the right reference): the reuse plan of
 * the paper executes a shared prefix once and resumes each task's suffix from
 * an EXACT boundary artifact (Sec. III-A "Execution", Sec. IV-B, Table II), so
 * its results must equal a per-task rerun from scratch (the fallback of
 * Sec. IV-B "Legality-aware handoff enforcement").  The oracle therefore is
 * that rerun, written out by definition: every task starts from |0...0>,
 * every gate of (prefix || suffix) is applied in order, no sharing, no fusion.
 *
 *   statevector: complex128, qubit q = bit q of the basis index.
 *   tableau    : Aaronson-Gottesman stabilizer tableau (the paper's
 *                stabilizer backend, Sec. III-A / Sec. V-B; tableau
 *                algorithm of its reference [aaronson2004stabilizer]),
 *                stored as UNPACKED bytes, one byte per bit.
 *
 * Conventions taken where the paper is silent:
 *   RX/RY/RZ(t) = exp(-i t P / 2); PHASE(t) = diag(1, e^{it});
 *   CPHASE(t) multiplies |11> by e^{it}; CNOT(q0 = control, q1 = target).
 *   Pauli term (c, x-mask m, z-mask z): P|x> = i^{#Y} (-1)^{popc(x&z)} |x^m>.
 *   Energy E = sum_k c_k <psi|P_k|psi> / <psi|psi>.
 *   Sampling: p_x = |psi_x|^2 / ||psi||^2, F_k = sum_{x<=k} p_x accumulated
 *   left to right in double; outcome of uniform u is min{k : F_k > u}, or the
 *   last x with p_x > 0 when rounding leaves u >= F_last.
 *   Tableau measurement of Z_a: pivot = smallest stabilizer row p with
 *   x_{p,a} = 1; a random outcome takes the bit carried by the gate record.
 *   RESET = measurement (outcome not recorded) followed by X when it was 1.
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* input records: must match the workload input format byte for byte */
typedef struct {
  uint32_t op, q0, q1, flags;
  double theta;
} orc_gate;

typedef struct {
  double coef;
  uint64_t xmask, zmask;
} orc_term;

enum {
  O_H = 1, O_X = 2, O_Y = 3, O_Z = 4, O_S = 5, O_SDG = 6, O_T = 7, O_TDG = 8,
  O_RX = 9, O_RY = 10, O_RZ = 11, O_PHASE = 12,
  O_CNOT = 20, O_CZ = 21, O_SWAP = 22, O_CPHASE = 23,
  O_MEASURE = 30, O_RESET = 31
};

/* ------------------------------------------------------------------------ */
/* statevector                                                              */
/* ------------------------------------------------------------------------ */

void orc_sv_zero(int n, cplx *psi) {
  size_t dim = (size_t)1 << n;
  for (size_t x = 0; x < dim; x++) psi[x] = 0.0;
  psi[0] = 1.0;
}

/* apply the 2x2 matrix [[u00,u01],[u10,u11]] to qubit q */
static void apply_1q(int n, cplx *psi, int q, cplx u00, cplx u01, cplx u10, cplx u11) {
  size_t dim = (size_t)1 << n, bit = (size_t)1 << q;
#pragma omp parallel for schedule(static)
  for (long long xx = 0; xx < (long long)dim; xx++) {
    size_t x = (size_t)xx;
    if (x & bit) continue;
    cplx a = psi[x], b = psi[x | bit];
    psi[x] = u00 * a + u01 * b;
    psi[x | bit] = u10 * a + u11 * b;
  }
}

static int gate_matrix_1q(const orc_gate *g, cplx *u00, cplx *u01, cplx *u10, cplx *u11) {
  double t = g->theta, c = cos(t / 2), s = sin(t / 2), r = 1.0 / sqrt(2.0);
  switch (g->op) {
    case O_H: *u00 = r; *u01 = r; *u10 = r; *u11 = -r; return 0;
    case O_X: *u00 = 0; *u01 = 1; *u10 = 1; *u11 = 0; return 0;
    case O_Y: *u00 = 0; *u01 = -I; *u10 = I; *u11 = 0; return 0;
    case O_Z: *u00 = 1; *u01 = 0; *u10 = 0; *u11 = -1; return 0;
    case O_S: *u00 = 1; *u01 = 0; *u10 = 0; *u11 = I; return 0;
    case O_SDG: *u00 = 1; *u01 = 0; *u10 = 0; *u11 = -I; return 0;
    case O_T: *u00 = 1; *u01 = 0; *u10 = 0; *u11 = cexp(I * (3.14159265358979323846 / 4)); return 0;
    case O_TDG: *u00 = 1; *u01 = 0; *u10 = 0; *u11 = cexp(-I * (3.14159265358979323846 / 4)); return 0;
    case O_RX: *u00 = c; *u01 = -I * s; *u10 = -I * s; *u11 = c; return 0;
    case O_RY: *u00 = c; *u01 = -s; *u10 = s; *u11 = c; return 0;
    case O_RZ: *u00 = cexp(-I * t / 2); *u01 = 0; *u10 = 0; *u11 = cexp(I * t / 2); return 0;
    case O_PHASE: *u00 = 1; *u01 = 0; *u10 = 0; *u11 = cexp(I * t); return 0;
    default: return -1;
  }
}

/* returns 0, or -1 on an unsupported/invalid gate */
int orc_sv_apply(int n, cplx *psi, const orc_gate *gates, size_t n_gates) {
  size_t dim = (size_t)1 << n;
  for (size_t k = 0; k < n_gates; k++) {
    const orc_gate *g = &gates[k];
    if (g->q0 >= (uint32_t)n) return -1;
    cplx u00, u01, u10, u11;
    if (gate_matrix_1q(g, &u00, &u01, &u10, &u11) == 0) {
      apply_1q(n, psi, (int)g->q0, u00, u01, u10, u11);
      continue;
    }
    if (g->q1 >= (uint32_t)n || g->q1 == g->q0) return -1;
    size_t a = (size_t)1 << g->q0, b = (size_t)1 << g->q1;
    switch (g->op) {
      case O_CNOT:
#pragma omp parallel for schedule(static)
        for (long long xx = 0; xx < (long long)dim; xx++) {
          size_t x = (size_t)xx;
          if ((x & a) && !(x & b)) { cplx t = psi[x]; psi[x] = psi[x | b]; psi[x | b] = t; }
        }
        break;
      case O_CZ:
#pragma omp parallel for schedule(static)
        for (long long xx = 0; xx < (long long)dim; xx++) {
          size_t x = (size_t)xx;
          if ((x & a) && (x & b)) psi[x] = -psi[x];
        }
        break;
      case O_CPHASE: {
        cplx ph = cexp(I * g->theta);
#pragma omp parallel for schedule(static)
        for (long long xx = 0; xx < (long long)dim; xx++) {
          size_t x = (size_t)xx;
          if ((x & a) && (x & b)) psi[x] *= ph;
        }
        break;
      }
      case O_SWAP:
#pragma omp parallel for schedule(static)
        for (long long xx = 0; xx < (long long)dim; xx++) {
          size_t x = (size_t)xx;
          if ((x & a) && !(x & b)) {
            size_t y = (x & ~a) | b;
            cplx t = psi[x]; psi[x] = psi[y]; psi[y] = t;
          }
        }
        break;
      default:
        return -1; /* MEASURE/RESET are not statevector operations here */
    }
  }
  return 0;
}

double orc_sv_norm2(int n, const cplx *psi) {
  size_t dim = (size_t)1 << n;
  double s = 0.0;
  for (size_t x = 0; x < dim; x++) s += creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
  return s;
}

static int popc64(uint64_t v) { return __builtin_popcountll(v); }

/* <psi|P|psi> for one Pauli term (complex; the imaginary part is ~0) */
void orc_sv_pauli_expect(int n, const cplx *psi, uint64_t m, uint64_t z,
                         double *re, double *im) {
  size_t dim = (size_t)1 << n;
  int ny = popc64(m & z);
  cplx iy = 1.0;
  for (int k = 0; k < (ny & 3); k++) iy *= I;
  cplx s = 0.0;
  for (size_t x = 0; x < dim; x++) {
    double sign = (popc64((uint64_t)x & z) & 1) ? -1.0 : 1.0;
    s += conj(psi[x ^ m]) * iy * sign * psi[x];
  }
  *re = creal(s);
  *im = cimag(s);
}

/* energy = sum_k c_k <P_k> / norm2 ; terms evaluated independently, summed in
 * term order */
int orc_sv_energy(int n, const cplx *psi, const orc_term *terms, size_t n_terms,
                  double *energy, double *norm2, double *per_term /* nullable */) {
  double *vals = (double *)malloc(sizeof(double) * (n_terms ? n_terms : 1));
  if (!vals) return -1;
#pragma omp parallel for schedule(dynamic, 1)
  for (long long k = 0; k < (long long)n_terms; k++) {
    double re, im;
    orc_sv_pauli_expect(n, psi, terms[k].xmask, terms[k].zmask, &re, &im);
    vals[k] = re;
  }
  double nrm = orc_sv_norm2(n, psi);
  double e = 0.0;
  for (size_t k = 0; k < n_terms; k++) {
    e += terms[k].coef * vals[k];
    if (per_term) per_term[k] = vals[k];
  }
  *energy = e / nrm;
  *norm2 = nrm;
  free(vals);
  return 0;
}

int orc_sv_sample(int n, const cplx *psi, const double *u, size_t shots, uint64_t *out) {
  size_t dim = (size_t)1 << n;
  double nrm = orc_sv_norm2(n, psi);
  double *F = (double *)malloc(sizeof(double) * dim);
  if (!F) return -1;
  double acc = 0.0;
  size_t last_nz = 0;
  for (size_t x = 0; x < dim; x++) {
    double p = (creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x])) / nrm;
    if (p > 0.0) last_nz = x;
    acc += p;
    F[x] = acc;
  }
  for (size_t s = 0; s < shots; s++) {
    /* min{k : F_k > u}: binary search over the non-decreasing F */
    size_t lo = 0, hi = dim; /* answer in [lo, hi) ; hi == dim means none */
    while (lo < hi) {
      size_t mid = lo + (hi - lo) / 2;
      if (F[mid] > u[s]) hi = mid; else lo = mid + 1;
    }
    out[s] = (lo < dim) ? (uint64_t)lo : (uint64_t)last_nz;
  }
  free(F);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* tableau (Aaronson-Gottesman), unpacked bytes                             */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n;
  uint8_t *x, *z, *r; /* (2n+1) x n, (2n+1) x n, (2n+1) */
} tab;

#define TX(t, i, j) ((t)->x[(size_t)(i) * (t)->n + (j)])
#define TZ(t, i, j) ((t)->z[(size_t)(i) * (t)->n + (j)])

static int tab_init(tab *t, int n) {
  t->n = n;
  size_t rows = 2 * (size_t)n + 1;
  t->x = (uint8_t *)calloc(rows * n, 1);
  t->z = (uint8_t *)calloc(rows * n, 1);
  t->r = (uint8_t *)calloc(rows, 1);
  if (!t->x || !t->z || !t->r) return -1;
  for (int i = 0; i < n; i++) {
    TX(t, i, i) = 1;     /* destabilizer i = X_i */
    TZ(t, n + i, i) = 1; /* stabilizer  i = Z_i */
  }
  return 0;
}

static void tab_free(tab *t) { free(t->x); free(t->z); free(t->r); }

/* exponent of i contributed by multiplying Pauli (x1,z1) onto (x2,z2) */
static int g_fn(int x1, int z1, int x2, int z2) {
  if (!x1 && !z1) return 0;
  if (x1 && z1) return z2 - x2;
  if (x1 && !z1) return z2 * (2 * x2 - 1);
  return x2 * (1 - 2 * z2);
}

/* row h <- row i * row h (Aaronson-Gottesman "rowsum") */
static void rowsum(tab *t, int h, int i) {
  int n = t->n;
  long sum = 2 * (long)t->r[h] + 2 * (long)t->r[i];
  for (int j = 0; j < n; j++) sum += g_fn(TX(t, i, j), TZ(t, i, j), TX(t, h, j), TZ(t, h, j));
  long m = ((sum % 4) + 4) % 4; /* 0 or 2 */
  t->r[h] = (m == 2);
  for (int j = 0; j < n; j++) {
    TX(t, h, j) ^= TX(t, i, j);
    TZ(t, h, j) ^= TZ(t, i, j);
  }
}

static void tab_cnot(tab *t, int a, int b) {
  int rows = 2 * t->n;
  for (int i = 0; i < rows; i++) {
    t->r[i] ^= TX(t, i, a) & TZ(t, i, b) & (TX(t, i, b) ^ TZ(t, i, a) ^ 1);
    TX(t, i, b) ^= TX(t, i, a);
    TZ(t, i, a) ^= TZ(t, i, b);
  }
}

static void tab_h(tab *t, int a) {
  int rows = 2 * t->n;
  for (int i = 0; i < rows; i++) {
    t->r[i] ^= TX(t, i, a) & TZ(t, i, a);
    uint8_t tmp = TX(t, i, a); TX(t, i, a) = TZ(t, i, a); TZ(t, i, a) = tmp;
  }
}

static void tab_s(tab *t, int a) {
  int rows = 2 * t->n;
  for (int i = 0; i < rows; i++) {
    t->r[i] ^= TX(t, i, a) & TZ(t, i, a);
    TZ(t, i, a) ^= TX(t, i, a);
  }
}

/* Pauli conjugations: X flips the sign of rows with a Z part on a, Z of rows
 * with an X part, Y of rows with exactly one of them. */
static void tab_pauli(tab *t, int a, int px, int pz) {
  int rows = 2 * t->n;
  for (int i = 0; i < rows; i++) t->r[i] ^= (px & TZ(t, i, a)) ^ (pz & TX(t, i, a));
}

static int tab_measure(tab *t, int a, int rand_bit) {
  int n = t->n;
  int p = -1;
  for (int i = n; i < 2 * n; i++)
    if (TX(t, i, a)) { p = i; break; }
  if (p >= 0) { /* random outcome */
    for (int i = 0; i < 2 * n; i++)
      if (i != p && TX(t, i, a)) rowsum(t, i, p);
    memcpy(&TX(t, p - n, 0), &TX(t, p, 0), n);
    memcpy(&TZ(t, p - n, 0), &TZ(t, p, 0), n);
    t->r[p - n] = t->r[p];
    memset(&TX(t, p, 0), 0, n);
    memset(&TZ(t, p, 0), 0, n);
    TZ(t, p, a) = 1;
    t->r[p] = (uint8_t)(rand_bit & 1);
    return t->r[p];
  }
  /* deterministic outcome: accumulate into scratch row 2n */
  int s = 2 * n;
  memset(&TX(t, s, 0), 0, n);
  memset(&TZ(t, s, 0), 0, n);
  t->r[s] = 0;
  for (int i = 0; i < n; i++)
    if (TX(t, i, a)) rowsum(t, s, i + n);
  return t->r[s];
}

/* Applies gates[0..n_gates) to the tableau t; outcomes as in orc_tab_run. */
static int tab_apply(tab *t, const orc_gate *gates, size_t n_gates, uint8_t *outcomes, size_t cap_out,
                     size_t *n_out) {
  const int n = t->n;
  size_t k_out = 0;
  int rc = 0;
  for (size_t k = 0; k < n_gates && rc == 0; k++) {
    const orc_gate *g = &gates[k];
    int a = (int)g->q0, b = (int)g->q1;
    if (a < 0 || a >= n) { rc = -1; break; }
    int two = (g->op == O_CNOT || g->op == O_CZ || g->op == O_SWAP);
    if (two && (b < 0 || b >= n || a == b)) { rc = -1; break; }
    switch (g->op) {
      case O_H: tab_h(t, a); break;
      case O_S: tab_s(t, a); break;
      case O_SDG: tab_s(t, a); tab_s(t, a); tab_s(t, a); break;
      case O_X: tab_pauli(t, a, 1, 0); break;
      case O_Y: tab_pauli(t, a, 1, 1); break;
      case O_Z: tab_pauli(t, a, 0, 1); break;
      case O_CNOT: tab_cnot(t, a, b); break;
      case O_CZ: tab_h(t, b); tab_cnot(t, a, b); tab_h(t, b); break;
      case O_SWAP: tab_cnot(t, a, b); tab_cnot(t, b, a); tab_cnot(t, a, b); break;
      case O_MEASURE: {
        int o = tab_measure(t, a, (int)g->theta);
        if (k_out >= cap_out) { rc = -3; break; }
        outcomes[k_out++] = (uint8_t)o;
        break;
      }
      case O_RESET: {
        int o = tab_measure(t, a, (int)g->theta);
        if (o) tab_pauli(t, a, 1, 0);
        break;
      }
      default: rc = -1;
    }
  }
  *n_out = k_out;
  return rc;
}

static void tab_export(const tab *t, uint8_t *x_out, uint8_t *z_out, uint8_t *r_out) {
  const size_t n = (size_t)t->n;
  memcpy(x_out, t->x, 2 * n * n);
  memcpy(z_out, t->z, 2 * n * n);
  memcpy(r_out, t->r, 2 * n);
}

/*
 * Runs a tableau circuit from |0...0>.  Writes the outcome of every MEASURE
 * (in order) to `outcomes` (capacity cap_out); *n_out = number of MEASURE ops.
 * If x_out/z_out/r_out are non-NULL they receive the final 2n rows (row-major
 * n bytes per row) and signs.  Returns 0, -1 on an invalid or non-Clifford
 * gate, -2 on allocation failure, -3 if the outcome buffer is too small.
 */
int orc_tab_run(int n, const orc_gate *gates, size_t n_gates, uint8_t *outcomes,
                size_t cap_out, size_t *n_out, uint8_t *x_out, uint8_t *z_out,
                uint8_t *r_out) {
  tab t;
  if (tab_init(&t, n)) { tab_free(&t); return -2; }
  int rc = tab_apply(&t, gates, n_gates, outcomes, cap_out, n_out);
  if (rc == 0 && x_out) tab_export(&t, x_out, z_out, r_out);
  tab_free(&t);
  return rc;
}

/*
 * The same algorithm continued from a given tableau: x_in/z_in/r_in are 2n
 * rows in the layout orc_tab_run exports (the rows of an earlier run), the
 * circuit is applied to them as orc_tab_run applies it to |0...0>.  The
 * algorithm is deterministic, so orc_tab_run(prefix || suffix) equals
 * orc_tab_run_from(rows after prefix, suffix) bit for bit (the outcomes of
 * the suffix and the final rows); test code uses it to check many tasks
 * that share one long prefix.
 */
int orc_tab_run_from(int n, const uint8_t *x_in, const uint8_t *z_in, const uint8_t *r_in,
                     const orc_gate *gates, size_t n_gates, uint8_t *outcomes, size_t cap_out,
                     size_t *n_out, uint8_t *x_out, uint8_t *z_out, uint8_t *r_out) {
  tab t;
  if (tab_init(&t, n)) { tab_free(&t); return -2; }
  memcpy(t.x, x_in, 2 * (size_t)n * n);
  memcpy(t.z, z_in, 2 * (size_t)n * n);
  memcpy(t.r, r_in, 2 * (size_t)n);
  int rc = tab_apply(&t, gates, n_gates, outcomes, cap_out, n_out);
  if (rc == 0 && x_out) tab_export(&t, x_out, z_out, r_out);
  tab_free(&t);
  return rc;
}

/* number of OpenMP threads the oracle's parallel loops use (1 without it) */
int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
