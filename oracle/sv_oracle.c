/*
 * Plain complex128 CPU oracle for the random-circuit state-vector method
 * (arXiv:1804.04797).  TEST INFRASTRUCTURE ONLY: it is called by the tests, by
 * smoke() and by the CPU-baseline legs of bench.py, never by the library.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * It is the numpy oracle (oracle/statevec.py) written in C so that 24..30-qubit cases
 * and the CPU timing run in reasonable time.  One gate = one full sweep:
 *   - one-qubit gate on qubit k: the pair update of §2,
 *       (alpha_i, alpha_{i+2^k}) <- [[a,b],[c,d]] (alpha_i, alpha_{i+2^k}), i_k = 0;
 *   - CZ on (a, b): alpha_i <- -alpha_i where bits a and b of i are both 1;
 *   - the projectors P0/P1 and Z are one-qubit matrices.
 * Amplitudes are interleaved (re, im) doubles, qubit k = bit k of the index.
 * The matrices follow the reading of the gate set: H = [[1,1],[1,-1]]/sqrt2,
 * T = diag(1, e^{i pi/4}), X^{1/2} = [[1+i,1-i],[1-i,1+i]]/2,
 * Y^{1/2} = [[1+i,-1-i],[1+i,1+i]]/2.
 *
 * oracle_branch_amplitudes follows the decomposition CZ = P0 (x) I + P1 (x) Z of §2
 * (Fig. 2 caption, Eq. 1): every CZ with one qubit in each half is expanded, half A
 * takes P_{l_j} on its qubit and half B takes Z^{l_j}; alpha_x is the sum over all
 * branches l of A_l[x_A] * B_l[x_B], summed in branch order (deterministic).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* gate kind codes of the interchange format */
enum { OK_H = 0, OK_T = 1, OK_SX = 2, OK_SY = 3, OK_CZ = 4, OK_P0 = 5, OK_P1 = 6, OK_Z = 7 };

/* m = {a, b, c, d} as (re, im) pairs */
static int one_qubit_matrix(int kind, int adjoint, double m[8]) {
  const double r = 1.0 / sqrt(2.0);
  double a_re = 0, a_im = 0, b_re = 0, b_im = 0, c_re = 0, c_im = 0, d_re = 0, d_im = 0;
  switch (kind) {
    case OK_H: a_re = r; b_re = r; c_re = r; d_re = -r; break;
    case OK_T: a_re = 1; d_re = cos(M_PI / 4); d_im = sin(M_PI / 4); break;
    case OK_SX:
      a_re = 0.5; a_im = 0.5; b_re = 0.5; b_im = -0.5;
      c_re = 0.5; c_im = -0.5; d_re = 0.5; d_im = 0.5; break;
    case OK_SY:
      a_re = 0.5; a_im = 0.5; b_re = -0.5; b_im = -0.5;
      c_re = 0.5; c_im = 0.5; d_re = 0.5; d_im = 0.5; break;
    case OK_P0: a_re = 1; break;
    case OK_P1: d_re = 1; break;
    case OK_Z: a_re = 1; d_re = -1; break;
    default: return -1;
  }
  if (adjoint) { /* conjugate transpose */
    double t_re = b_re, t_im = b_im;
    b_re = c_re; b_im = -c_im; c_re = t_re; c_im = -t_im;
    a_im = -a_im; d_im = -d_im;
  }
  m[0] = a_re; m[1] = a_im; m[2] = b_re; m[3] = b_im;
  m[4] = c_re; m[5] = c_im; m[6] = d_re; m[7] = d_im;
  return 0;
}

static void pair_update(double *psi, int n, int k, const double *m, int parallel) {
  const int64_t pairs = (int64_t)1 << (n - 1);
  const int64_t low = ((int64_t)1 << k) - 1;
  const int64_t stride = (int64_t)1 << k;
#pragma omp parallel for schedule(static) if (parallel)
  for (int64_t p = 0; p < pairs; ++p) {
    const int64_t i0 = ((p & ~low) << 1) | (p & low);
    const int64_t i1 = i0 + stride;
    const double xr = psi[2 * i0], xi = psi[2 * i0 + 1];
    const double yr = psi[2 * i1], yi = psi[2 * i1 + 1];
    psi[2 * i0] = m[0] * xr - m[1] * xi + m[2] * yr - m[3] * yi;
    psi[2 * i0 + 1] = m[0] * xi + m[1] * xr + m[2] * yi + m[3] * yr;
    psi[2 * i1] = m[4] * xr - m[5] * xi + m[6] * yr - m[7] * yi;
    psi[2 * i1 + 1] = m[4] * xi + m[5] * xr + m[6] * yi + m[7] * yr;
  }
}

static void cz_update(double *psi, int n, int a, int b, int parallel) {
  const int64_t size = (int64_t)1 << n;
#pragma omp parallel for schedule(static) if (parallel)
  for (int64_t i = 0; i < size; ++i) {
    if (((i >> a) & 1) && ((i >> b) & 1)) {
      psi[2 * i] = -psi[2 * i];
      psi[2 * i + 1] = -psi[2 * i + 1];
    }
  }
}

static int apply_list(double *psi, int n, size_t ngates, const uint8_t *kind,
                      const uint8_t *q0, const uint8_t *q1, int adjoint, int parallel) {
  for (size_t s = 0; s < ngates; ++s) {
    const size_t g = adjoint ? ngates - 1 - s : s;
    if (q0[g] >= n) return -2;
    if (kind[g] == OK_CZ) {
      if (q1[g] >= n || q1[g] == q0[g]) return -2;
      cz_update(psi, n, q0[g], q1[g], parallel);
    } else {
      double m[8];
      if (one_qubit_matrix(kind[g], adjoint, m)) return -3;
      pair_update(psi, n, q0[g], m, parallel);
    }
  }
  return 0;
}

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* Apply the gate list (or its inverse when adjoint != 0) to psi in place. */
int oracle_run(int n, size_t ngates, const uint8_t *kind, const uint8_t *q0,
               const uint8_t *q1, int adjoint, double *psi) {
  if (n < 1 || n > 40) return -1;
  return apply_list(psi, n, ngates, kind, q0, q1, adjoint, 1);
}

static uint64_t compress_bits(uint64_t x, const int *qubits, int count) {
  uint64_t out = 0;
  for (int j = 0; j < count; ++j) out |= ((x >> qubits[j]) & 1ull) << j;
  return out;
}

/* Amplitudes alpha_x for m bitstrings by the cut decomposition.  out: 2*m doubles. */
int oracle_branch_amplitudes(int n, size_t ngates, const uint8_t *kind, const uint8_t *q0,
                             const uint8_t *q1, uint64_t half_a_mask, size_t m,
                             const uint64_t *bits, double *out) {
  if (n < 2 || n > 64) return -1;
  int qa[64], qb[64], local[64], side[64];
  int na = 0, nb = 0;
  for (int q = 0; q < n; ++q) {
    if ((half_a_mask >> q) & 1) { side[q] = 0; local[q] = na; qa[na++] = q; }
    else { side[q] = 1; local[q] = nb; qb[nb++] = q; }
  }
  if (na < 1 || nb < 1 || na > 30 || nb > 30) return -1;
  /* per-half gate lists; kind 255 marks a cut placeholder whose q1 holds the cut index */
  uint8_t *ka = malloc(ngates), *a0 = malloc(ngates), *a1 = malloc(ngates);
  uint8_t *kb = malloc(ngates), *b0 = malloc(ngates), *b1 = malloc(ngates);
  size_t ga = 0, gb = 0;
  int t = 0;
  for (size_t g = 0; g < ngates; ++g) {
    if (kind[g] == OK_CZ) {
      const int sa = side[q0[g]], sb = side[q1[g]];
      if (sa == sb) {
        if (sa == 0) { ka[ga] = OK_CZ; a0[ga] = local[q0[g]]; a1[ga] = local[q1[g]]; ++ga; }
        else { kb[gb] = OK_CZ; b0[gb] = local[q0[g]]; b1[gb] = local[q1[g]]; ++gb; }
      } else {
        const int qa_side = sa == 0 ? q0[g] : q1[g];
        const int qb_side = sa == 0 ? q1[g] : q0[g];
        ka[ga] = 255; a0[ga] = local[qa_side]; a1[ga] = (uint8_t)t; ++ga;
        kb[gb] = 255; b0[gb] = local[qb_side]; b1[gb] = (uint8_t)t; ++gb;
        ++t;
      }
    } else if (side[q0[g]] == 0) {
      ka[ga] = kind[g]; a0[ga] = local[q0[g]]; a1[ga] = 0; ++ga;
    } else {
      kb[gb] = kind[g]; b0[gb] = local[q0[g]]; b1[gb] = 0; ++gb;
    }
  }
  if (t > 24) { free(ka); free(a0); free(a1); free(kb); free(b0); free(b1); return -1; }
  const int64_t branches = (int64_t)1 << t;
  double *contrib = calloc((size_t)branches * m * 2, sizeof(double));
  int status = 0;
#pragma omp parallel
  {
    double *A = malloc(sizeof(double) * 2 * ((size_t)1 << na));
    double *B = malloc(sizeof(double) * 2 * ((size_t)1 << nb));
    uint8_t *kk = malloc(ngates + 1), *k0 = malloc(ngates + 1), *k1 = malloc(ngates + 1);
#pragma omp for schedule(dynamic, 1)
    for (int64_t l = 0; l < branches; ++l) {
      for (int h = 0; h < 2; ++h) {
        const int nh = h == 0 ? na : nb;
        double *S = h == 0 ? A : B;
        const uint8_t *hk = h == 0 ? ka : kb, *h0 = h == 0 ? a0 : b0, *h1 = h == 0 ? a1 : b1;
        const size_t hg = h == 0 ? ga : gb;
        size_t cnt = 0;
        for (size_t g = 0; g < hg; ++g) {
          if (hk[g] != 255) { kk[cnt] = hk[g]; k0[cnt] = h0[g]; k1[cnt] = h1[g]; ++cnt; continue; }
          const int lj = (int)((l >> h1[g]) & 1);
          if (h == 0) { kk[cnt] = lj ? OK_P1 : OK_P0; k0[cnt] = h0[g]; k1[cnt] = 0; ++cnt; }
          else if (lj) { kk[cnt] = OK_Z; k0[cnt] = h0[g]; k1[cnt] = 0; ++cnt; }
        }
        memset(S, 0, sizeof(double) * 2 * ((size_t)1 << nh));
        S[0] = 1.0;
        if (apply_list(S, nh, cnt, kk, k0, k1, 0, 0)) status = -3;
      }
      for (size_t j = 0; j < m; ++j) {
        const uint64_t xa = compress_bits(bits[j], qa, na), xb = compress_bits(bits[j], qb, nb);
        const double ar = A[2 * xa], ai = A[2 * xa + 1], br = B[2 * xb], bi = B[2 * xb + 1];
        contrib[2 * ((size_t)l * m + j)] = ar * br - ai * bi;
        contrib[2 * ((size_t)l * m + j) + 1] = ar * bi + ai * br;
      }
    }
    free(A); free(B); free(kk); free(k0); free(k1);
  }
  for (size_t j = 0; j < m; ++j) {
    double sr = 0, si = 0;
    for (int64_t l = 0; l < branches; ++l) {
      sr += contrib[2 * ((size_t)l * m + j)];
      si += contrib[2 * ((size_t)l * m + j) + 1];
    }
    out[2 * j] = sr; out[2 * j + 1] = si;
  }
  free(contrib); free(ka); free(a0); free(a1); free(kb); free(b0); free(b1);
  return status;
}

/* sum |alpha|^2 and sum |alpha|^4 over the state, fp64. */
void oracle_reductions(int n, const double *psi, double *norm2, double *sum_p2) {
  const int64_t size = (int64_t)1 << n;
  double s2 = 0, s4 = 0;
#pragma omp parallel for reduction(+ : s2, s4) schedule(static)
  for (int64_t i = 0; i < size; ++i) {
    const double p = psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
    s2 += p;
    s4 += p * p;
  }
  *norm2 = s2;
  *sum_p2 = s4;
}
