/*
 * FP64 CPU oracle for the general dense tensor contraction
 *
 *     C[c] := alpha * sum_{k in K} A[a(c,k)] * B[b(c,k)] + beta * C[c]
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the tests, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header or constant
 * with the CUDA path.
 *
 * What it computes (the plain definition, written out):
 *   The paper asks for tensor computations that reduce to level-3 products
 *   without explicit conversion between tensors and matrices (Sec. 1,
 *   "Challenges", tensor item; Sec. 2.3 "Supporting tensor computations",
 *   block-scatter item) over arbitrarily strided layouts (Girder 2, data
 *   layout goal).  The operation itself is Einstein summation over labels:
 *     - a label in C and in exactly one of A, B is a free index;
 *     - a label in A and B but not in C is summed over;
 *     - a label in A, B and C is a batch index (free, shared by all three).
 *   Element addresses are data + sum_i index_i * stride_i (strides in
 *   elements), so transposition is a change of strides (Sec. 2.1,
 *   "Variations on functionality").
 *   alpha == 0: A and B are not read.  beta == 0: C is not read (a NaN in
 *   C is overwritten).  An empty contracted extent gives C := beta*C.
 *
 * How: one loop over every entry of C (an odometer over C's modes), and for
 * each an inner odometer over the contracted multi-index with an fma per
 * term, in fp64.  No blocking, fusion or reordering.  Threads (pthreads)
 * split the flat range of C entries; each entry is still a plain serial sum.
 *
 * oracle_entries() evaluates chosen entries only, either with the same
 * plain sum or with the compensated dot product Dot2 of Ogita, Rump and
 * Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005,
 * Algorithm 5.3): TwoProduct by fma and TwoSum (Knuth) carried along the
 * sum, giving a result as accurate as if computed in twice the working
 * precision.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXDIM 16

enum {
  OR_OK = 0,
  OR_ERR_ARG = -1,
  OR_ERR_LABEL = -2,
  OR_ERR_EXTENT = -3,
};

typedef struct {
  int nfree;                /* modes of C */
  int64_t fext[OR_MAXDIM];  /* extent of each C mode */
  int64_t fsa[OR_MAXDIM];   /* stride of that label in A (0 if absent) */
  int64_t fsb[OR_MAXDIM];   /* stride in B (0 if absent) */
  int64_t fsc[OR_MAXDIM];   /* stride in C */
  int nsum;                 /* contracted labels */
  int64_t sext[OR_MAXDIM];
  int64_t ssa[OR_MAXDIM];
  int64_t ssb[OR_MAXDIM];
  int64_t nC;               /* number of entries of C */
  int64_t nK;               /* number of terms per entry */
} or_problem;

static int find_label(int n, const int32_t* lab, int32_t x) {
  for (int i = 0; i < n; ++i)
    if (lab[i] == x) return i;
  return -1;
}

static int has_repeat(int n, const int32_t* lab) {
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (lab[i] == lab[j]) return 1;
  return 0;
}

/* Sort the labels into free (in C) and contracted (in A and B, not in C). */
static int or_classify(int ndA, const int64_t* eA, const int64_t* sA, const int32_t* lA,
                       int ndB, const int64_t* eB, const int64_t* sB, const int32_t* lB,
                       int ndC, const int64_t* eC, const int64_t* sC, const int32_t* lC,
                       or_problem* p) {
  if (ndA < 0 || ndB < 0 || ndC < 0 || ndA > OR_MAXDIM || ndB > OR_MAXDIM || ndC > OR_MAXDIM)
    return OR_ERR_ARG;
  if (has_repeat(ndA, lA) || has_repeat(ndB, lB) || has_repeat(ndC, lC)) return OR_ERR_LABEL;
  memset(p, 0, sizeof(*p));
  p->nC = 1;
  for (int i = 0; i < ndC; ++i) {
    int ia = find_label(ndA, lA, lC[i]);
    int ib = find_label(ndB, lB, lC[i]);
    if (ia < 0 && ib < 0) return OR_ERR_LABEL; /* C label with no source */
    if (eC[i] < 0) return OR_ERR_ARG;
    if (ia >= 0 && eA[ia] != eC[i]) return OR_ERR_EXTENT;
    if (ib >= 0 && eB[ib] != eC[i]) return OR_ERR_EXTENT;
    p->fext[p->nfree] = eC[i];
    p->fsc[p->nfree] = sC[i];
    p->fsa[p->nfree] = ia >= 0 ? sA[ia] : 0;
    p->fsb[p->nfree] = ib >= 0 ? sB[ib] : 0;
    p->nfree++;
    p->nC *= eC[i];
  }
  p->nK = 1;
  for (int i = 0; i < ndA; ++i) {
    if (eA[i] < 0) return OR_ERR_ARG;
    if (find_label(ndC, lC, lA[i]) >= 0) continue;
    int ib = find_label(ndB, lB, lA[i]);
    if (ib < 0) return OR_ERR_LABEL; /* label in A only */
    if (eB[ib] != eA[i]) return OR_ERR_EXTENT;
    p->sext[p->nsum] = eA[i];
    p->ssa[p->nsum] = sA[i];
    p->ssb[p->nsum] = sB[ib];
    p->nsum++;
    p->nK *= eA[i];
  }
  for (int i = 0; i < ndB; ++i) {
    if (eB[i] < 0) return OR_ERR_ARG;
    if (find_label(ndC, lC, lB[i]) < 0 && find_label(ndA, lA, lB[i]) < 0)
      return OR_ERR_LABEL; /* label in B only */
  }
  return OR_OK;
}

/* Offsets of C entry number `flat` (first C mode varies fastest). */
static void or_decode(const or_problem* p, int64_t flat, int64_t idx[OR_MAXDIM],
                      int64_t* oa, int64_t* ob, int64_t* oc) {
  *oa = *ob = *oc = 0;
  for (int i = 0; i < p->nfree; ++i) {
    idx[i] = p->fext[i] ? flat % p->fext[i] : 0;
    flat = p->fext[i] ? flat / p->fext[i] : 0;
    *oa += idx[i] * p->fsa[i];
    *ob += idx[i] * p->fsb[i];
    *oc += idx[i] * p->fsc[i];
  }
}

/* Plain fp64 sum over the contracted multi-index (first label fastest). */
static double or_sum_plain(const or_problem* p, const double* A, const double* B,
                           int64_t oa, int64_t ob) {
  int64_t k[OR_MAXDIM];
  double acc = 0.0;
  if (p->nK == 0) return 0.0;
  for (int i = 0; i < p->nsum; ++i) k[i] = 0;
  for (int64_t t = 0; t < p->nK; ++t) {
    acc = fma(A[oa], B[ob], acc);
    for (int i = 0; i < p->nsum; ++i) { /* odometer step */
      oa += p->ssa[i];
      ob += p->ssb[i];
      if (++k[i] < p->sext[i]) break;
      oa -= p->ssa[i] * p->sext[i];
      ob -= p->ssb[i] * p->sext[i];
      k[i] = 0;
    }
  }
  return acc;
}

/* Dot2 (Ogita-Rump-Oishi 2005, Alg. 5.3): the sum as if in doubled precision. */
static double or_sum_dot2(const or_problem* p, const double* A, const double* B,
                          int64_t oa, int64_t ob) {
  int64_t k[OR_MAXDIM];
  double s = 0.0, c = 0.0;
  if (p->nK == 0) return 0.0;
  for (int i = 0; i < p->nsum; ++i) k[i] = 0;
  for (int64_t t = 0; t < p->nK; ++t) {
    double x = A[oa], y = B[ob];
    double h = x * y;
    double r = fma(x, y, -h);   /* TwoProduct: x*y == h + r exactly */
    double s1 = s + h;          /* TwoSum(s, h) = (s1, q) */
    double z = s1 - s;
    double q = (s - (s1 - z)) + (h - z);
    s = s1;
    c += q + r;
    for (int i = 0; i < p->nsum; ++i) {
      oa += p->ssa[i];
      ob += p->ssb[i];
      if (++k[i] < p->sext[i]) break;
      oa -= p->ssa[i] * p->sext[i];
      ob -= p->ssb[i] * p->sext[i];
      k[i] = 0;
    }
  }
  return s + c;
}

typedef struct {
  const or_problem* p;
  double alpha, beta;
  const double *A, *B;
  double* C;
  int64_t lo, hi;
} or_job;

static void* or_worker(void* arg) {
  or_job* j = (or_job*)arg;
  const or_problem* p = j->p;
  int64_t idx[OR_MAXDIM];
  for (int64_t f = j->lo; f < j->hi; ++f) {
    int64_t oa, ob, oc;
    or_decode(p, f, idx, &oa, &ob, &oc);
    double v = 0.0;
    if (j->alpha != 0.0) v = j->alpha * or_sum_plain(p, j->A, j->B, oa, ob);
    if (j->beta != 0.0) v += j->beta * j->C[oc];
    j->C[oc] = v;
  }
  return NULL;
}

/*
 * Full contraction, in place on C.  Strides are in elements and may be any
 * non-negative values; the caller passes base pointers of fp64 buffers.
 * Returns 0, or a negative code for malformed label sets or extents.
 */
int oracle_contract(double alpha,
                    int ndA, const int64_t* eA, const int64_t* sA, const int32_t* lA, const double* A,
                    int ndB, const int64_t* eB, const int64_t* sB, const int32_t* lB, const double* B,
                    double beta,
                    int ndC, const int64_t* eC, const int64_t* sC, const int32_t* lC, double* C,
                    int nthreads) {
  or_problem p;
  int rc = or_classify(ndA, eA, sA, lA, ndB, eB, sB, lB, ndC, eC, sC, lC, &p);
  if (rc) return rc;
  if (p.nC == 0) return OR_OK;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > p.nC) nthreads = (int)p.nC;
  pthread_t th[256];
  or_job jobs[256];
  int64_t per = (p.nC + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].p = &p;
    jobs[t].alpha = alpha;
    jobs[t].beta = beta;
    jobs[t].A = A;
    jobs[t].B = B;
    jobs[t].C = C;
    jobs[t].lo = (int64_t)t * per;
    jobs[t].hi = jobs[t].lo + per < p.nC ? jobs[t].lo + per : p.nC;
    if (jobs[t].lo > jobs[t].hi) jobs[t].lo = jobs[t].hi;
  }
  for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, or_worker, &jobs[t]);
  or_worker(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  return OR_OK;
}

/*
 * Selected entries only.  `cidx` holds n rows of ndC multi-indices (one per
 * C mode, in C's mode order).  out[i] = alpha*sum + beta*Cin[entry] where
 * Cin is read only when beta != 0.  mode 0: plain fp64 sum; mode 1: Dot2.
 */
int oracle_entries(double alpha,
                   int ndA, const int64_t* eA, const int64_t* sA, const int32_t* lA, const double* A,
                   int ndB, const int64_t* eB, const int64_t* sB, const int32_t* lB, const double* B,
                   double beta,
                   int ndC, const int64_t* eC, const int64_t* sC, const int32_t* lC, const double* Cin,
                   int64_t n, const int64_t* cidx, int mode, double* out) {
  or_problem p;
  int rc = or_classify(ndA, eA, sA, lA, ndB, eB, sB, lB, ndC, eC, sC, lC, &p);
  if (rc) return rc;
  for (int64_t s = 0; s < n; ++s) {
    int64_t oa = 0, ob = 0, oc = 0;
    for (int i = 0; i < ndC; ++i) {
      int64_t x = cidx[s * ndC + i];
      if (x < 0 || x >= p.fext[i]) return OR_ERR_ARG;
      oa += x * p.fsa[i];
      ob += x * p.fsb[i];
      oc += x * p.fsc[i];
    }
    double v = 0.0;
    if (alpha != 0.0)
      v = alpha * (mode == 1 ? or_sum_dot2(&p, A, B, oa, ob) : or_sum_plain(&p, A, B, oa, ob));
    if (beta != 0.0) v += beta * Cin[oc];
    out[s] = v;
  }
  return OR_OK;
}
