/*
 * SRLA oracle -- a plain, slow, single-threaded CPU restatement of the sliding-window
 * super point cardinality estimator (SRLA, arXiv 1803.10369).
 *
 * TEST INFRASTRUCTURE ONLY.  This file exists to check the CUDA library against the
 * paper.  Only the test suite, the package smoke check and the benchmark's CPU-baseline
 * leg may load it; the product path never does.  It shares no code, header or constant
 * with the CUDA library.
 *
 * Representation: every distance recorder (DR, Section 3.2) is held literally as its
 * distance d in [0, 2^z - 1] (one uint16 per recorder), initialised to 2^z - 1, set to 0
 * by DRset and incremented by DRslide over the whole array at every slice end
 * (Algorithm 3).  No stamps, no fusion, no reordering.
 *
 * Readings of the paper this file takes (each is listed with its reason in the design
 * notes of the repository):
 *   R1  hash functions: the family is not given; each role uses its own member
 *       h(x) = (a*x + b) mod (2^61 - 1) of the polynomial family, low 32 bits, and an
 *       index into m (a power of two) cells is h & (m - 1).  Roles: rows 0..u-1 (RH_i on
 *       aip), u = SLE cell (on bip), u+1 = SRE cell (on bip), u+2 = sampling (on bip).
 *   R2  sampling follows the text of Section 3.2: a pair updates the SRE iff
 *       LSB(H(bip)) >= tau, with LSB(0) taken as 32.
 *   R3  UnionSE (Algorithm 1) joins with DRjoin = max; the join starts from 0 (the
 *       identity of max), so a union cell is inside the window iff it is inside the window
 *       in every row.
 *   R4  the candidate rule is order free: a host sampled in slice T becomes a new
 *       candidate iff its union SRE at the end of T holds >= ceil(rho*g) in-window cells.
 *       Duplicates are removed exactly (sort + unique) instead of with the SI bits.
 *   R5  Eq. 9 edges: w <= g'*UP gives 0; w == g' (or UP == 1) gives +infinity, flagged
 *       saturated; the super point test is est >= theta (Definition 2).
 *   R6  carried hosts (Algorithm 3) join the next slice's candidate list unconditionally.
 *  R11  inline mode (orc_set_inline): the candidate test of Algorithm 2 as printed, run at
 *       packet time after the SRE update, with the 16 super point indicator bits SI of
 *       Section 4.1 suppressing repeats.  The SI bit of a host is chosen from aip (the paper
 *       names H3(aip), H4(aip) and H4(bip) in different places; hashing bip would let one
 *       host in many times): bits 28..31 of the sampling-role hash applied to aip.  The
 *       threshold is ceil(rho*g) as in R4.  SI is cleared at every slice end and set again
 *       for the carried hosts (Algorithm 3).  The result depends on packet order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_P61 ((((uint64_t)1) << 61) - 1)
#define ORC_MAX_ROWS 16

/* Report flags (an interface shared by convention only; the CUDA library defines its own). */
#define ORC_SUPER 1u
#define ORC_SATURATED 2u
#define ORC_CARRIED 4u
#define ORC_NEW 8u

typedef struct orc {
  uint32_t u, v, g, gl, z, k, theta;
  uint64_t ha[ORC_MAX_ROWS + 3], hb[ORC_MAX_ROWS + 3];
  uint32_t dmax;  /* 2^z - 1: "never seen / too old" (Section 3.2) */
  int tau;        /* Eq. 1 */
  uint32_t rho_g; /* ceil(rho * g) */
  uint64_t T;     /* index of the open slice */
  uint16_t *re;   /* SRE recorders RE[i][c][j], u*v*g */
  uint16_t *le;   /* SLE recorders LE[i][c][j], u*v*gl */
  uint32_t *s;    /* hosts of pairs sampled into the SRE in the open slice */
  size_t ns, caps;
  uint32_t *carry; /* NCSIP of the previous slice end (Algorithm 3), ascending */
  size_t ncarry;
  /* inline mode (R11) */
  int inline_mode;
  uint16_t *si;     /* SI[i][c]: 16 super point indicator bits per estimator */
  uint32_t *ins;    /* hosts inserted into CSIP by the scan in the open slice */
  size_t nins, capins;
  /* results of the last slice end */
  uint64_t cnt[ORC_MAX_ROWS];
  double up;
  size_t nsu, nnew, nrep;
  uint32_t *rep_aip, *rep_w, *rep_flags;
  double *rep_est;
} orc;

/* ---------------------------------------------------------------- definitions ---- */

/* Definition of LSB (Section 3.2): index of the first 1 bit counted from the right. */
int orc_lsb(uint32_t x) {
  if (x == 0) return 32; /* R2: no 1 bit at all */
  int i = 0;
  while ((x & 1u) == 0) {
    x >>= 1;
    i++;
  }
  return i;
}

/* Eq. 1: tau = ceil(log2(theta / g)), clamped at 0 when theta < g. */
int orc_tau(uint32_t theta, uint32_t g) {
  double t = ceil(log2((double)theta / (double)g));
  return t < 0 ? 0 : (int)t;
}

/* Section 3.2: rho = 0.99 * (1 - e^{-1/3}). */
double orc_rho(void) { return 0.99 * (1.0 - exp(-1.0 / 3.0)); }

/* The SRE detection threshold rho*g as a whole number of recorders. */
uint32_t orc_rho_g(uint32_t g) { return (uint32_t)ceil(orc_rho() * (double)g); }

/* R1: member (a, b) of the polynomial family, evaluated by its definition. */
uint32_t orc_hash_ab(uint64_t a, uint64_t b, uint32_t x) {
  unsigned __int128 t = (unsigned __int128)a * (unsigned __int128)x + (unsigned __int128)b;
  return (uint32_t)(uint64_t)(t % (unsigned __int128)ORC_P61);
}

uint32_t orc_hash(const orc *o, int role, uint32_t x) { return orc_hash_ab(o->ha[role], o->hb[role], x); }

/* Eq. 9 with the edge rules of R5.  w may be fractional so the algebra can be checked. */
double orc_estimate(uint32_t gl, double up, double w, uint32_t *flags) {
  double g = (double)gl;
  *flags = 0;
  if (w >= g || up >= 1.0) {
    *flags = ORC_SATURATED;
    return INFINITY;
  }
  if (w <= g * up) return 0.0;
  return -g * log(1.0 - (w - g * up) / (g * (1.0 - up)));
}

/* ------------------------------------------------------------------ lifecycle ---- */

orc *orc_create(uint32_t u, uint32_t v, uint32_t g, uint32_t gl, uint32_t z, uint32_t k,
                uint32_t theta, const uint64_t *ha, const uint64_t *hb, uint64_t start_slice) {
  if (u < 1 || u > ORC_MAX_ROWS || z < 1 || z > 16 || k < 1 || k > ((1u << z) - 1)) return NULL;
  if (v == 0 || g == 0 || gl == 0 || (v & (v - 1)) || (g & (g - 1)) || (gl & (gl - 1))) return NULL;
  orc *o = (orc *)calloc(1, sizeof(orc));
  if (!o) return NULL;
  o->u = u; o->v = v; o->g = g; o->gl = gl; o->z = z; o->k = k; o->theta = theta;
  for (uint32_t r = 0; r < u + 3; r++) {
    o->ha[r] = ha[r];
    o->hb[r] = hb[r];
  }
  o->dmax = (1u << z) - 1;
  o->tau = orc_tau(theta, g);
  o->rho_g = orc_rho_g(g);
  o->T = start_slice;
  size_t nre = (size_t)u * v * g, nle = (size_t)u * v * gl;
  o->re = (uint16_t *)malloc(nre * sizeof(uint16_t));
  o->le = (uint16_t *)malloc(nle * sizeof(uint16_t));
  if (!o->re || !o->le) {
    free(o->re); free(o->le); free(o);
    return NULL;
  }
  /* DRinit (Section 3.2): every recorder starts at 2^z - 1. */
  for (size_t i = 0; i < nre; i++) o->re[i] = (uint16_t)o->dmax;
  for (size_t i = 0; i < nle; i++) o->le[i] = (uint16_t)o->dmax;
  return o;
}

static void orc_free_report(orc *o) {
  free(o->rep_aip); free(o->rep_w); free(o->rep_flags); free(o->rep_est);
  o->rep_aip = o->rep_w = o->rep_flags = NULL;
  o->rep_est = NULL;
  o->nrep = 0;
}

void orc_destroy(orc *o) {
  if (!o) return;
  orc_free_report(o);
  free(o->re); free(o->le); free(o->s); free(o->carry); free(o->si); free(o->ins);
  free(o);
}

/* R11: the SI bit of host aip. */
static uint32_t si_index(const orc *o, uint32_t aip) { return orc_hash(o, (int)o->u + 2, aip) >> 28; }

/* Set the SI bit of aip in each of its u estimators. */
static void si_mark(orc *o, uint32_t aip) {
  uint32_t b = si_index(o, aip);
  for (uint32_t i = 0; i < o->u; i++) {
    uint32_t c = orc_hash(o, (int)i, aip) & (o->v - 1);
    o->si[(size_t)i * o->v + c] |= (uint16_t)(1u << b);
  }
}

/* Switch to the inline candidate test (R11) before the first packet; the SI bits start
   clear, then hold the bits of the carried hosts.  Returns 0, or -1 without memory. */
int orc_set_inline(orc *o, int on) {
  o->inline_mode = on ? 1 : 0;
  if (!on) return 0;
  if (!o->si) {
    o->si = (uint16_t *)calloc((size_t)o->u * o->v, sizeof(uint16_t));
    if (!o->si) return -1;
  }
  memset(o->si, 0, (size_t)o->u * o->v * sizeof(uint16_t));
  for (size_t x = 0; x < o->ncarry; x++) si_mark(o, o->carry[x]);
  return 0;
}

static size_t re_at(const orc *o, uint32_t i, uint32_t c, uint32_t j) {
  return ((size_t)i * o->v + c) * o->g + j;
}
static size_t le_at(const orc *o, uint32_t i, uint32_t c, uint32_t j) {
  return ((size_t)i * o->v + c) * o->gl + j;
}

uint32_t orc_ure_count(const orc *o, uint32_t aip, uint32_t limit);

/* -------------------------------------------------------------- the scan ---------- */

/* Algorithm 2 (ScanIPpair) for every pair, under readings R1, R2 and R4. */
int orc_push(orc *o, const uint32_t *pairs, size_t n) {
  for (size_t p = 0; p < n; p++) {
    uint32_t aip = pairs[2 * p], bip = pairs[2 * p + 1];
    /* DRset on the SLE recorder selected by bip in each of the u estimators of aip. */
    uint32_t jl = orc_hash(o, (int)o->u, bip) & (o->gl - 1);
    for (uint32_t i = 0; i < o->u; i++) {
      uint32_t c = orc_hash(o, (int)i, aip) & (o->v - 1);
      o->le[le_at(o, i, c, jl)] = 0;
    }
    /* Sampling by the least significant bit of a hash of bip (Section 3.2). */
    if (orc_lsb(orc_hash(o, (int)o->u + 2, bip)) >= o->tau) {
      uint32_t jr = orc_hash(o, (int)o->u + 1, bip) & (o->g - 1);
      for (uint32_t i = 0; i < o->u; i++) {
        uint32_t c = orc_hash(o, (int)i, aip) & (o->v - 1);
        o->re[re_at(o, i, c, jr)] = 0;
      }
      if (o->ns == o->caps) {
        size_t nc = o->caps ? 2 * o->caps : 1024;
        uint32_t *ns = (uint32_t *)realloc(o->s, nc * sizeof(uint32_t));
        if (!ns) return -1;
        o->s = ns;
        o->caps = nc;
      }
      o->s[o->ns++] = aip;
      if (o->inline_mode) {
        /* Algorithm 2: the host is tested by its union SRE right after the update, and
           inserted into CSIP unless its SI bit is already set in all u estimators. */
        if (orc_ure_count(o, aip, o->k) >= o->rho_g) {
          uint32_t b = si_index(o, aip);
          uint16_t usi = 0xFFFFu; /* USI: AND over the rows (Algorithm 1) */
          for (uint32_t i = 0; i < o->u; i++) {
            uint32_t c = orc_hash(o, (int)i, aip) & (o->v - 1);
            usi &= o->si[(size_t)i * o->v + c];
          }
          if (!((usi >> b) & 1u)) {
            if (o->nins == o->capins) {
              size_t nc = o->capins ? 2 * o->capins : 256;
              uint32_t *ni = (uint32_t *)realloc(o->ins, nc * sizeof(uint32_t));
              if (!ni) return -1;
              o->ins = ni;
              o->capins = nc;
            }
            o->ins[o->nins++] = aip;
            si_mark(o, aip);
          }
        }
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------- union estimator counts ---- */

/* |URE(aip)|^k of Algorithm 1 (R3): SRE cells whose joined distance is below `limit`. */
uint32_t orc_ure_count(const orc *o, uint32_t aip, uint32_t limit) {
  uint32_t col[ORC_MAX_ROWS];
  for (uint32_t i = 0; i < o->u; i++) col[i] = orc_hash(o, (int)i, aip) & (o->v - 1);
  uint32_t cnt = 0;
  for (uint32_t j = 0; j < o->g; j++) {
    uint32_t joined = 0; /* identity of max */
    for (uint32_t i = 0; i < o->u; i++) {
      uint32_t d = o->re[re_at(o, i, col[i], j)];
      if (d > joined) joined = d; /* DRjoin */
    }
    if (joined < limit) cnt++;
  }
  return cnt;
}

/* |ULE(aip)|^k of Algorithm 1 (R3). */
uint32_t orc_ule_count(const orc *o, uint32_t aip, uint32_t limit) {
  uint32_t col[ORC_MAX_ROWS];
  for (uint32_t i = 0; i < o->u; i++) col[i] = orc_hash(o, (int)i, aip) & (o->v - 1);
  uint32_t cnt = 0;
  for (uint32_t j = 0; j < o->gl; j++) {
    uint32_t joined = 0;
    for (uint32_t i = 0; i < o->u; i++) {
      uint32_t d = o->le[le_at(o, i, col[i], j)];
      if (d > joined) joined = d;
    }
    if (joined < limit) cnt++;
  }
  return cnt;
}

/* ------------------------------------------------------------ the slice end ------- */

static int cmp_u32(const void *a, const void *b) {
  uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
  return (x > y) - (x < y);
}

static size_t sort_unique(uint32_t *a, size_t n) {
  if (n == 0) return 0;
  qsort(a, n, sizeof(uint32_t), cmp_u32);
  size_t m = 1;
  for (size_t i = 1; i < n; i++)
    if (a[i] != a[m - 1]) a[m++] = a[i];
  return m;
}

/*
 * End of slice T: Section 4.2 (row census, Eq. 8, Eq. 9 over the candidate list) and
 * Algorithm 3 (slide every recorder, carry the candidates that still pass the SRE test).
 * Returns the number of report entries, or -1 when memory runs out.
 */
long orc_end_slice(orc *o) {
  const uint32_t u = o->u, v = o->v, g = o->g, gl = o->gl, k = o->k;

  /* |LDR(i)|^k: SLE recorders of row i inside the window (Section 4.2). */
  for (uint32_t i = 0; i < u; i++) {
    uint64_t c = 0;
    for (size_t x = 0; x < (size_t)v * gl; x++)
      if (o->le[(size_t)i * v * gl + x] < k) c++;
    o->cnt[i] = c;
  }
  /* Eq. 8: UP = prod_i |LDR(i)|^k / (g' v). */
  double up = 1.0;
  for (uint32_t i = 0; i < u; i++) up *= (double)o->cnt[i] / ((double)gl * (double)v);
  o->up = up;

  /* New candidates (R4): sampled hosts of this slice passing the union SRE test now.  In
     inline mode (R11) they are the hosts the scan inserted. */
  size_t nsu = sort_unique(o->s, o->ns);
  o->nsu = nsu;
  uint32_t *newc = (uint32_t *)malloc(((nsu > o->nins ? nsu : o->nins) + 1) * sizeof(uint32_t));
  if (!newc) return -1;
  size_t nnew = 0;
  if (o->inline_mode) {
    for (size_t x = 0; x < o->nins; x++) newc[nnew++] = o->ins[x];
    nnew = sort_unique(newc, nnew);
  } else {
    for (size_t x = 0; x < nsu; x++)
      if (orc_ure_count(o, o->s[x], k) >= o->rho_g) newc[nnew++] = o->s[x];
  }
  o->nnew = nnew;

  /* Candidate list: union of the new candidates and the carried list (R6), ascending. */
  orc_free_report(o);
  size_t cap = nnew + o->ncarry;
  o->rep_aip = (uint32_t *)malloc((cap ? cap : 1) * sizeof(uint32_t));
  o->rep_w = (uint32_t *)malloc((cap ? cap : 1) * sizeof(uint32_t));
  o->rep_flags = (uint32_t *)malloc((cap ? cap : 1) * sizeof(uint32_t));
  o->rep_est = (double *)malloc((cap ? cap : 1) * sizeof(double));
  if (!o->rep_aip || !o->rep_w || !o->rep_flags || !o->rep_est) {
    free(newc);
    return -1;
  }
  size_t a = 0, b = 0, n = 0;
  while (a < nnew || b < o->ncarry) {
    uint32_t x;
    uint32_t f = 0;
    if (b >= o->ncarry || (a < nnew && newc[a] < o->carry[b])) {
      x = newc[a++];
      f = ORC_NEW;
    } else if (a >= nnew || o->carry[b] < newc[a]) {
      x = o->carry[b++];
      f = ORC_CARRIED;
    } else {
      x = newc[a++];
      b++;
      f = ORC_NEW | ORC_CARRIED;
    }
    o->rep_aip[n] = x;
    o->rep_flags[n] = f;
    n++;
  }
  o->nrep = n;
  free(newc);

  /* Eq. 9 for every candidate, from its union SLE (Algorithm 1). */
  for (size_t x = 0; x < n; x++) {
    uint32_t w = orc_ule_count(o, o->rep_aip[x], k);
    uint32_t ef;
    double est = orc_estimate(gl, up, (double)w, &ef);
    uint32_t f = o->rep_flags[x] | ef;
    if ((ef & ORC_SATURATED) || est >= (double)o->theta) f |= ORC_SUPER;
    o->rep_w[x] = w;
    o->rep_est[x] = est;
    o->rep_flags[x] = f;
  }

  /* Algorithm 3: clear every SI (inline mode), DRslide on every recorder of the SRE and
     SLE arrays. */
  if (o->inline_mode) memset(o->si, 0, (size_t)u * v * sizeof(uint16_t));
  for (size_t x = 0; x < (size_t)u * v * g; x++)
    if (o->re[x] < o->dmax) o->re[x]++;
  for (size_t x = 0; x < (size_t)u * v * gl; x++)
    if (o->le[x] < o->dmax) o->le[x]++;

  /* Algorithm 3: the candidates still passing the SRE test after the slide are carried. */
  free(o->carry);
  o->carry = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
  if (!o->carry) return -1;
  o->ncarry = 0;
  for (size_t x = 0; x < n; x++)
    if (orc_ure_count(o, o->rep_aip[x], k) >= o->rho_g) {
      o->carry[o->ncarry++] = o->rep_aip[x];
      if (o->inline_mode) si_mark(o, o->rep_aip[x]);
    }

  o->ns = 0;
  o->nins = 0;
  o->T++;
  return (long)n;
}

/* ------------------------------------------------------------- accessors ---------- */

void orc_get_report(const orc *o, uint32_t *aip, uint32_t *w, double *est, uint32_t *flags) {
  for (size_t x = 0; x < o->nrep; x++) {
    aip[x] = o->rep_aip[x];
    w[x] = o->rep_w[x];
    est[x] = o->rep_est[x];
    flags[x] = o->rep_flags[x];
  }
}

void orc_get_census(const orc *o, uint64_t *cnt, double *up, uint64_t *sizes) {
  for (uint32_t i = 0; i < o->u; i++) cnt[i] = o->cnt[i];
  *up = o->up;
  sizes[0] = o->nsu;
  sizes[1] = o->nnew;
  sizes[2] = o->nrep;
  sizes[3] = o->ncarry;
}

uint64_t orc_slice(const orc *o) { return o->T; }
int orc_tau_of(const orc *o) { return o->tau; }
uint32_t orc_rho_g_of(const orc *o) { return o->rho_g; }
size_t orc_n_carry(const orc *o) { return o->ncarry; }

void orc_get_carry(const orc *o, uint32_t *out) {
  for (size_t x = 0; x < o->ncarry; x++) out[x] = o->carry[x];
}

void orc_get_state(const orc *o, uint16_t *re, uint16_t *le) {
  memcpy(re, o->re, (size_t)o->u * o->v * o->g * sizeof(uint16_t));
  memcpy(le, o->le, (size_t)o->u * o->v * o->gl * sizeof(uint16_t));
}

/* Pending sampled hosts of the open slice (with repeats), for tests. */
size_t orc_n_sampled(const orc *o) { return o->ns; }
void orc_get_sampled(const orc *o, uint32_t *out) {
  for (size_t x = 0; x < o->ns; x++) out[x] = o->s[x];
}

/* Restore a literal state (checkpoint tests): distances, open slice, carried list. */
int orc_set_state(orc *o, const uint16_t *re, const uint16_t *le, uint64_t T,
                  const uint32_t *carry, size_t ncarry) {
  memcpy(o->re, re, (size_t)o->u * o->v * o->g * sizeof(uint16_t));
  memcpy(o->le, le, (size_t)o->u * o->v * o->gl * sizeof(uint16_t));
  o->T = T;
  free(o->carry);
  o->carry = (uint32_t *)malloc((ncarry ? ncarry : 1) * sizeof(uint32_t));
  if (!o->carry) return -1;
  memcpy(o->carry, carry, ncarry * sizeof(uint32_t));
  o->ncarry = ncarry;
  o->ns = 0;
  o->nins = 0;
  return o->inline_mode ? orc_set_inline(o, 1) : 0;
}

/* The SI bits (inline mode), u*v uint16. */
void orc_get_si(const orc *o, uint16_t *out) {
  if (o->si) memcpy(out, o->si, (size_t)o->u * o->v * sizeof(uint16_t));
}

/* Hash a batch of values with one role (tests build brute-force sets from it). */
void orc_hash_many(const orc *o, int role, const uint32_t *x, size_t n, uint32_t *out) {
  for (size_t i = 0; i < n; i++) out[i] = orc_hash(o, role, x[i]);
}
