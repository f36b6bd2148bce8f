/*
 * RecSplit oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, sequential CPU implementation of RecSplit (Esposito, Mueller Graf,
 * Vigna, "RecSplit: Minimal Perfect Hashing via Recursive Splitting").  It is
 * the reference the CUDA library is compared against, bit for bit.  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it; the library never calls it and shares no source with it.
 *
 * Every step follows the paper's order:
 *   fingerprint (Sec. 6.1)  ->  bucket by fixed-point inversion (Sec. 6.1)
 *   ->  per bucket, recursive splitting tree in preorder (Sec. 4, Sec. 5.4)
 *   ->  Golomb-Rice codes, all fixed parts then all unary parts (Sec. 6.2)
 *   ->  double Elias-Fano of prefix sums and offsets (Sec. 6.3, Sec. 7.4)
 *   ->  lookup by descending the tree (Sec. 4, Sec. 6.2).
 * The choices the paper leaves open (hash family, bit conventions, Elias-Fano
 * details) are fixed as listed in the design notes of the repository; each
 * function below states the reading it implements.  Floating point appears
 * only in the Golomb-Rice parameter table (Eq. gr with Eq. probsplit), as in
 * the paper.
 *
 * The optional thread count of orc_build_* splits the buckets over POSIX
 * threads; buckets are independent (Sec. 4), so the bytes do not depend on it.
 *
 * The *_e functions also build the perfect, non-minimal variant the paper's
 * conclusion leaves for future work (enlarged bijection codomains): with leaf
 * range extra e > 0 a leaf of m >= 2 keys maps its keys injectively into
 * [0, m + e) and everything downstream counts output ranges instead of keys
 * (header word 2 holds the leaf size | e << 8).  e = 0 is the minimal
 * structure, byte for byte.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

#define ORC_OK 0
#define ORC_E_INVALID (-1)
#define ORC_E_DUPLICATE (-2)
#define ORC_E_SEARCH_LIMIT (-4)
#define ORC_E_NOMEM (-5)

#define ORC_MAGIC 0x31544C5053434552ULL /* "RECSPLT1" */
#define ORC_HEADER_WORDS 16
#define ORC_MAX_TRIALS (1ULL << 36)
#define ORC_WEYL 0x9E3779B97F4A7C15ULL
#define ORC_FP_HI 0x6A09E667F3BCC909ULL
#define ORC_FP_LO 0xBB67AE8584CAA73BULL
#define ORC_INV_HI 14 /* one 64-bit anchor every 2^14 ones */
#define ORC_INV_LO 8  /* one 16-bit offset every 2^8 ones  */
#define ORC_MAX_FANOUT 64

/* ------------------------------------------------------------------ */
/* Mixer: the splitmix64 finalizer (Steele, Lea, Flood, OOPSLA 2014).  */
/* ------------------------------------------------------------------ */
uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Sec. 6.1: every key becomes a 128-bit signature (hi, lo).  For a 64-bit
 * key each half is the mixer of the key xored with its own constant, so the
 * signature (and each half) is injective in the key. */
void orc_fingerprint_u64(const uint64_t* keys, uint64_t n, uint64_t* hi, uint64_t* lo) {
  for (uint64_t i = 0; i < n; i++) {
    hi[i] = orc_mix64(keys[i] ^ ORC_FP_HI);
    lo[i] = orc_mix64(keys[i] ^ ORC_FP_LO);
  }
}

/* Sec. 6.1 for byte strings: the bytes are read as little-endian 64-bit words
 * (last word zero-padded); two chains absorb the words, the second one with
 * the word's halves swapped, and the length is folded in at the end so that
 * zero padding cannot make two strings equal. */
void orc_fingerprint_one_bytes(const uint8_t* p, uint64_t len, uint64_t* hi, uint64_t* lo) {
  uint64_t a = ORC_FP_HI, c = ORC_FP_LO;
  for (uint64_t pos = 0; pos < len; pos += 8) {
    uint64_t w = 0;
    for (uint64_t k = 0; k < 8 && pos + k < len; k++) w |= (uint64_t)p[pos + k] << (8 * k);
    uint64_t wswap = (w >> 32) | (w << 32);
    a = orc_mix64(a ^ w);
    c = orc_mix64(c ^ wswap);
  }
  *hi = orc_mix64(a + len);
  *lo = orc_mix64(c + len);
}

void orc_fingerprint_bytes(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, uint64_t* hi,
                           uint64_t* lo) {
  for (uint64_t i = 0; i < n; i++)
    orc_fingerprint_one_bytes(bytes + offsets[i], offsets[i + 1] - offsets[i], &hi[i], &lo[i]);
}

/* Sec. 4 / Sec. 6.1: bucket = floor(hi * N / 2^64), N = ceil(n / b). */
uint64_t orc_bucket(uint64_t hi, uint64_t nbuckets) { return (uint64_t)(((u128)hi * nbuckets) >> 64); }

/* ------------------------------------------------------------------ */
/* Hash family phi^m_i (Sec. 4), avoiding correlation (Sec. 7.3).      */
/* ------------------------------------------------------------------ */
/* Function number i at depth d is keyed by (i * 64 + d) times the Weyl
 * constant, so functions at different depths of one root-to-leaf path are
 * never the same.  It acts on the lower signature half only (the upper half
 * chose the bucket): the key is xored in and the first two xorshift-multiply
 * rounds of the splitmix64 finalizer are applied (its last xorshift would only
 * touch the lowest of the 32 bits kept).  The range reduction to [0, m) is
 * fixed-point multiplication of the top 32 bits, as the paper uses for
 * buckets. */
uint32_t orc_phi(uint64_t lo, uint32_t depth, uint64_t index, uint64_t m) {
  uint64_t key = ((index << 6) | depth) * ORC_WEYL;
  uint64_t z = lo ^ key;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return (uint32_t)(((z >> 32) * m) >> 32);
}

/* ------------------------------------------------------------------ */
/* Splitting strategy (Sec. 5.4).                                      */
/* ------------------------------------------------------------------ */
/* Lower aggregation s = max(2, ceil(0.35 l + 0.5)) and upper aggregation
 * t = ceil(0.21 l + 0.9) for l >= 7, else 2, both evaluated exactly in
 * integers: 0.35 l + 0.5 = (7 l + 10) / 20 and 0.21 l + 0.9 = (21 l + 90) / 100. */
static uint64_t orc_lower_aggr(uint32_t leaf) {
  uint64_t s = (7ULL * leaf + 10 + 19) / 20;
  return s < 2 ? 2 : s;
}
static uint64_t orc_upper_aggr(uint32_t leaf) {
  if (leaf < 7) return 2;
  return (21ULL * leaf + 90 + 99) / 100;
}

/* Parts of a node with m > leaf keys, in the order of the codomain: the
 * split unit u is l for m <= s*l, s*l for m <= s*t*l, and above that the
 * split is binary with a left part of ceil(floor(m/2) / (s*t*l)) * s*t*l
 * keys.  All parts have u keys except the last.  Returns the fanout, or 0
 * for a leaf (m <= l).  *unit gets u (the left part for binary splits). */
int orc_strategy(uint32_t leaf, uint64_t m, uint64_t* unit, uint64_t* parts, int cap) {
  if (m <= leaf) return 0;
  uint64_t s = orc_lower_aggr(leaf), t = orc_upper_aggr(leaf);
  uint64_t u;
  int fanout;
  if (m <= s * leaf) {
    u = leaf;
  } else if (m <= s * t * leaf) {
    u = s * leaf;
  } else {
    /* above the second aggregation level the fanout is fixed at 2 */
    uint64_t big = s * t * leaf;
    u = ((m / 2 + big - 1) / big) * big;
    if (cap < 2) return -1;
    parts[0] = u;
    parts[1] = m - u;
    *unit = u;
    return 2;
  }
  fanout = (int)((m + u - 1) / u);
  if (fanout > cap) return -1;
  for (int j = 0; j < fanout - 1; j++) parts[j] = u;
  parts[fanout - 1] = m - u * (uint64_t)(fanout - 1);
  *unit = u;
  return fanout;
}

/* ------------------------------------------------------------------ */
/* Golomb-Rice parameters (Sec. 5.4 Eq. gr, Sec. 7.2) and skip tables. */
/* ------------------------------------------------------------------ */
/* ln of the success probability of one trial at a node of size m:
 * leaves m!/m^m (Sec. 5.2), splits Eq. probsplit (Sec. 5.1).  With leaf
 * range extra e > 0 (the perfect, non-minimal variant the conclusion of the
 * paper sketches: the codomain of a leaf of m keys is enlarged to R = m + e)
 * a leaf trial succeeds when the m values are distinct in [0, R):
 * R! / ((R - m)! R^m).  e = 0 gives m!/m^m. */
double orc_log_success_e(uint32_t leaf, uint32_t extra, uint64_t m) {
  double dm = (double)m;
  if (m <= leaf) {
    double dr = (double)(m + extra);
    return lgamma(dr + 1.0) - lgamma(dr - dm + 1.0) - dm * log(dr);
  }
  double lp = lgamma(dm + 1.0) - dm * log(dm);
  uint64_t parts[ORC_MAX_FANOUT], u;
  int f = orc_strategy(leaf, m, &u, parts, ORC_MAX_FANOUT);
  for (int j = 0; j < f; j++) {
    double k = (double)parts[j];
    lp += k * log(k) - lgamma(k + 1.0);
  }
  return lp;
}

double orc_log_success(uint32_t leaf, uint64_t m) { return orc_log_success_e(leaf, 0, m); }

/* The real number whose ceiling (clamped at 0) is the parameter of Eq. gr:
 * lg(-lg(phi) / lg(1 - p)) = lg(ln(phi) / -ln(1 - p)). */
double orc_golomb_rice_x_e(uint32_t leaf, uint32_t extra, uint64_t m) {
  double p = exp(orc_log_success_e(leaf, extra, m));
  double golden = (1.0 + sqrt(5.0)) / 2.0;
  return log2(log(golden) / -log1p(-p));
}

double orc_golomb_rice_x(uint32_t leaf, uint64_t m) { return orc_golomb_rice_x_e(leaf, 0, m); }

/* floor(lg x) for x >= 1, and 0 for x = 0 (lambda of Sec. 2). */
static int orc_lambda(uint64_t x) {
  int k = -1;
  while (x) {
    x >>= 1;
    k++;
  }
  return k < 0 ? 0 : k;
}

/* Golomb-Rice parameter of a node with m keys.  For m < 2^16 it is Eq. gr
 * evaluated in double; larger (split) nodes use the integer approximation of
 * Sec. 7.2, with ">>" read as a right shift as Sec. 7.1 uses it. */
int orc_golomb_rice_e(uint32_t leaf, uint32_t extra, uint64_t m) {
  if (m <= 1) return 0;
  if (m < 65536) {
    double x = orc_golomb_rice_x_e(leaf, extra, m);
    int r = (int)ceil(x);
    return r < 0 ? 0 : r;
  }
  uint64_t parts[ORC_MAX_FANOUT], u;
  int f = orc_strategy(leaf, m, &u, parts, ORC_MAX_FANOUT);
  int64_t acc = (int64_t)(((uint64_t)(f - 1) * 5) >> 1);
  for (int j = 0; j < f; j++) acc += orc_lambda(parts[j] + (parts[j] >> 1));
  acc -= orc_lambda(m);
  if (acc < 0) acc = 0;
  return (int)(acc >> 1);
}

int orc_golomb_rice(uint32_t leaf, uint64_t m) { return orc_golomb_rice_e(leaf, 0, m); }

typedef struct {
  uint32_t leaf;
  uint32_t extra;  /* leaf range extra e (0: minimal)                */
  uint64_t mmax;
  int* r;          /* Golomb-Rice parameter per node size            */
  uint64_t* fbits; /* fixed bits of the subtree of a node of size m  */
  uint64_t* codes; /* number of codes (indices) in that subtree      */
  uint64_t* rng;   /* output range of that subtree: the sum of its leaves' ranges
                      (m + e for a leaf of m >= 2 keys, m for 0 or 1 key) */
} orc_tables;

static void orc_tables_free(orc_tables* t) {
  free(t->r);
  free(t->fbits);
  free(t->codes);
  free(t->rng);
}

/* Sec. 6.2 skip information: for every size m the fixed bits and the number
 * of codes of a whole subtree.  Sizes 0 and 1 carry no code (Fig. 1). */
static int orc_tables_init(orc_tables* t, uint32_t leaf, uint32_t extra, uint64_t mmax) {
  t->leaf = leaf;
  t->extra = extra;
  t->mmax = mmax;
  t->r = calloc(mmax + 1, sizeof(int));
  t->fbits = calloc(mmax + 1, sizeof(uint64_t));
  t->codes = calloc(mmax + 1, sizeof(uint64_t));
  t->rng = calloc(mmax + 1, sizeof(uint64_t));
  if (!t->r || !t->fbits || !t->codes || !t->rng) {
    orc_tables_free(t);
    return ORC_E_NOMEM;
  }
  t->rng[0] = 0;
  if (mmax >= 1) t->rng[1] = 1;
  for (uint64_t m = 2; m <= mmax; m++) {
    t->r[m] = orc_golomb_rice_e(leaf, extra, m);
    t->fbits[m] = (uint64_t)t->r[m];
    t->codes[m] = 1;
    t->rng[m] = m + extra;
    if (m > leaf) {
      uint64_t parts[ORC_MAX_FANOUT], u;
      int f = orc_strategy(leaf, m, &u, parts, ORC_MAX_FANOUT);
      t->rng[m] = 0;
      for (int j = 0; j < f; j++) {
        t->fbits[m] += t->fbits[parts[j]];
        t->codes[m] += t->codes[parts[j]];
        t->rng[m] += t->rng[parts[j]];
      }
    }
    /* a bucket's size is read back from its range, so the range must grow
     * strictly with the size; this is checked for every size */
    if (t->rng[m] <= t->rng[m - 1]) {
      orc_tables_free(t);
      return ORC_E_INVALID;
    }
  }
  return ORC_OK;
}

/* The node size whose subtree has output range R, or UINT64_MAX. */
static uint64_t orc_size_of_range(const orc_tables* t, uint64_t R) {
  uint64_t a = 0, b = t->mmax;
  while (a < b) {
    uint64_t mid = (a + b + 1) / 2;
    if (t->rng[mid] <= R)
      a = mid;
    else
      b = mid - 1;
  }
  return t->rng[a] == R ? a : UINT64_MAX;
}

/* Output range of the subtree of a node of m keys with leaf range extra e
 * (m itself for e = 0), or 0 if the tables cannot be made. */
uint64_t orc_node_range(uint32_t leaf, uint32_t extra, uint64_t m) {
  orc_tables t;
  if (orc_tables_init(&t, leaf, extra, m < 2 ? 2 : m)) return 0;
  uint64_t r = t.rng[m];
  orc_tables_free(&t);
  return r;
}

int orc_skip(uint32_t leaf, uint64_t m, uint64_t* fixed_bits, uint64_t* codes) {
  orc_tables t;
  if (orc_tables_init(&t, leaf, 0, m < 2 ? 2 : m)) return ORC_E_NOMEM;
  *fixed_bits = m < 2 ? 0 : t.fbits[m];
  *codes = m < 2 ? 0 : t.codes[m];
  orc_tables_free(&t);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Brute-force searches (Sec. 4).                                      */
/* ------------------------------------------------------------------ */
/* First i such that phi^R_i maps the m keys of a leaf to m distinct values
 * of [0, R): for R = m a bijection onto [0, m) (Sec. 4), for R > m an
 * injection (the perfect, non-minimal variant).  R <= 64. */
int64_t orc_leaf_seed_range(const uint64_t* lo, uint64_t m, uint64_t R, uint32_t depth, uint64_t cap) {
  for (uint64_t i = 0; i < cap; i++) {
    uint64_t seen = 0;
    int ok = 1;
    for (uint64_t j = 0; j < m; j++) {
      uint64_t bit = 1ULL << orc_phi(lo[j], depth, i, R);
      if (seen & bit) {
        ok = 0; /* two keys on one value: not a bijection */
        break;
      }
      seen |= bit;
    }
    if (ok) return (int64_t)i;
  }
  return -1;
}

int64_t orc_leaf_seed(const uint64_t* lo, uint64_t m, uint32_t depth, uint64_t cap) {
  return orc_leaf_seed_range(lo, m, m, depth, cap);
}

/* First i such that, mapping the m keys to [0, m) with phi^m_i, exactly k_t
 * keys land in the t-th interval [k_0 + ... + k_{t-1}, k_0 + ... + k_t) for
 * every t < s - 1 (the last part then holds the rest). */
int64_t orc_split_seed(const uint64_t* lo, uint64_t m, uint32_t depth, uint32_t leaf, uint64_t cap) {
  uint64_t parts[ORC_MAX_FANOUT], bounds[ORC_MAX_FANOUT + 1], count[ORC_MAX_FANOUT], u;
  int f = orc_strategy(leaf, m, &u, parts, ORC_MAX_FANOUT);
  if (f <= 0) return -1;
  bounds[0] = 0;
  for (int t = 0; t < f; t++) bounds[t + 1] = bounds[t] + parts[t];
  for (uint64_t i = 0; i < cap; i++) {
    memset(count, 0, sizeof(count));
    for (uint64_t j = 0; j < m; j++) {
      uint64_t v = orc_phi(lo[j], depth, i, m);
      int t = 0;
      while (v >= bounds[t + 1]) t++;
      count[t]++;
    }
    int ok = 1;
    for (int t = 0; t < f - 1; t++)
      if (count[t] != parts[t]) ok = 0;
    if (ok) return (int64_t)i;
  }
  return -1;
}

/* ------------------------------------------------------------------ */
/* One bucket: the splitting tree in preorder (Sec. 4).                */
/* ------------------------------------------------------------------ */
/* Writes the indices of the tree of the m keys in preorder into seeds[],
 * advancing *pos; the keys array is reordered (children become contiguous).
 * tmp must hold m words. */
static int orc_solve(const orc_tables* t, uint64_t* keys, uint64_t m, uint32_t depth, uint64_t* tmp,
                     uint64_t* seeds, uint64_t* sizes, uint64_t* pos) {
  if (m <= 1) return ORC_OK;
  if (depth > 63) return ORC_E_INVALID;
  if (m <= t->leaf) {
    int64_t s = orc_leaf_seed_range(keys, m, m + t->extra, depth, ORC_MAX_TRIALS);
    if (s < 0) return ORC_E_SEARCH_LIMIT;
    seeds[*pos] = (uint64_t)s;
    sizes[*pos] = m;
    (*pos)++;
    return ORC_OK;
  }
  int64_t s = orc_split_seed(keys, m, depth, t->leaf, ORC_MAX_TRIALS);
  if (s < 0) return ORC_E_SEARCH_LIMIT;
  seeds[*pos] = (uint64_t)s;
  sizes[*pos] = m;
  (*pos)++;
  uint64_t parts[ORC_MAX_FANOUT], u, start[ORC_MAX_FANOUT + 1], fill[ORC_MAX_FANOUT];
  int f = orc_strategy(t->leaf, m, &u, parts, ORC_MAX_FANOUT);
  start[0] = 0;
  for (int j = 0; j < f; j++) {
    start[j + 1] = start[j] + parts[j];
    fill[j] = 0;
  }
  for (uint64_t j = 0; j < m; j++) {
    uint64_t v = orc_phi(keys[j], depth, (uint64_t)s, m);
    int p = 0;
    while (v >= start[p + 1]) p++;
    tmp[start[p] + fill[p]++] = keys[j];
  }
  memcpy(keys, tmp, m * sizeof(uint64_t));
  for (int j = 0; j < f; j++) {
    int rc = orc_solve(t, keys + start[j], parts[j], depth + 1, tmp, seeds, sizes, pos);
    if (rc) return rc;
  }
  return ORC_OK;
}

static int orc_cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y);
}

/* Preorder indices of one bucket given the lower signature halves of its
 * keys.  Keys sharing their lower half can never be separated (Sec. 7.3
 * works on the lower half only), so they are reported as duplicates. */
int orc_bucket_seeds_from_keys_e(const uint64_t* lo, uint64_t m, uint32_t leaf, uint32_t extra, uint64_t* seeds,
                                 uint64_t* count) {
  if (leaf < 1 || leaf > 24 || leaf + extra > 32) return ORC_E_INVALID;
  uint64_t* keys = malloc((m + 1) * sizeof(uint64_t));
  uint64_t* tmp = malloc((m + 1) * sizeof(uint64_t));
  uint64_t* sizes = malloc((m + 1) * sizeof(uint64_t));
  orc_tables t;
  int rc = ORC_E_NOMEM;
  if (!keys || !tmp || !sizes || orc_tables_init(&t, leaf, extra, m < 2 ? 2 : m)) goto out_nomem;
  memcpy(keys, lo, m * sizeof(uint64_t));
  qsort(keys, m, sizeof(uint64_t), orc_cmp_u64);
  rc = ORC_OK;
  for (uint64_t j = 1; j < m; j++)
    if (keys[j] == keys[j - 1]) rc = ORC_E_DUPLICATE;
  *count = 0;
  if (rc == ORC_OK) rc = orc_solve(&t, keys, m, 0, tmp, seeds, sizes, count);
  orc_tables_free(&t);
out_nomem:
  free(keys);
  free(tmp);
  free(sizes);
  return rc;
}

int orc_bucket_seeds_from_keys(const uint64_t* lo, uint64_t m, uint32_t leaf, uint64_t* seeds, uint64_t* count) {
  return orc_bucket_seeds_from_keys_e(lo, m, leaf, 0, seeds, count);
}

/* ------------------------------------------------------------------ */
/* Bit arrays: bit k is bit (k mod 64) of word k / 64.                 */
/* ------------------------------------------------------------------ */
static void orc_put_bits(uint64_t* w, uint64_t pos, uint64_t val, int width) {
  for (int k = 0; k < width; k++)
    if ((val >> k) & 1) w[(pos + k) >> 6] |= 1ULL << ((pos + k) & 63);
}
static uint64_t orc_get_bits(const uint64_t* w, uint64_t pos, int width) {
  uint64_t v = 0;
  for (int k = 0; k < width; k++) v |= ((w[(pos + k) >> 6] >> ((pos + k) & 63)) & 1ULL) << k;
  return v;
}
static int orc_get_bit(const uint64_t* w, uint64_t pos) { return (int)((w[pos >> 6] >> (pos & 63)) & 1); }

/* ------------------------------------------------------------------ */
/* Whole build.                                                        */
/* ------------------------------------------------------------------ */
typedef struct {
  const orc_tables* t;
  const uint64_t* sorted_lo; /* keys grouped by bucket */
  const uint64_t* bstart;    /* prefix sums s_i, N + 1 entries */
  const uint64_t* cbase;     /* first code slot of each bucket  */
  uint64_t* seeds;           /* code slots, preorder per bucket */
  uint64_t* sizes;
  uint64_t b0, b1;
  int rc;
} orc_job;

static void* orc_worker(void* arg) {
  orc_job* j = (orc_job*)arg;
  uint64_t mmax = j->t->mmax;
  uint64_t* keys = malloc((mmax + 1) * sizeof(uint64_t));
  uint64_t* tmp = malloc((mmax + 1) * sizeof(uint64_t));
  j->rc = ORC_OK;
  if (!keys || !tmp) j->rc = ORC_E_NOMEM;
  for (uint64_t b = j->b0; b < j->b1 && j->rc == ORC_OK; b++) {
    uint64_t m = j->bstart[b + 1] - j->bstart[b];
    memcpy(keys, j->sorted_lo + j->bstart[b], m * sizeof(uint64_t));
    qsort(keys, m, sizeof(uint64_t), orc_cmp_u64);
    for (uint64_t k = 1; k < m; k++)
      if (keys[k] == keys[k - 1]) j->rc = ORC_E_DUPLICATE;
    if (j->rc) break;
    uint64_t pos = 0;
    j->rc = orc_solve(j->t, keys, m, 0, tmp, j->seeds + j->cbase[b], j->sizes + j->cbase[b], &pos);
  }
  free(keys);
  free(tmp);
  return NULL;
}

/* Elias-Fano lower width: max(0, floor(lg(u / count))) with integer lg. */
static int orc_ef_width(uint64_t u, uint64_t count) {
  uint64_t q = u / count;
  return q ? orc_lambda(q) : 0;
}

static uint64_t orc_words(uint64_t bits) { return (bits + 63) / 64; }

/* Sections of the serialized structure, in order (all 64-bit words). */
typedef struct {
  uint64_t tree, lower, upper_a, upper_b, anchors, subs, total;
  uint64_t n_anchor, n_sub;
} orc_layout;

static void orc_layout_of(const uint64_t* h, orc_layout* L) {
  uint64_t nb = h[4], T = h[5], la = h[10], lb = h[11], ua = h[12], ub = h[13];
  L->n_anchor = (nb >> ORC_INV_HI) + 1;
  L->n_sub = (nb >> ORC_INV_LO) + 1;
  L->tree = ORC_HEADER_WORDS;
  L->lower = L->tree + orc_words(T);
  L->upper_a = L->lower + orc_words((nb + 1) * (la + lb));
  L->upper_b = L->upper_a + orc_words(ua);
  L->anchors = L->upper_b + orc_words(ub);
  L->subs = L->anchors + 2 * L->n_anchor;
  L->total = L->subs + (2 * L->n_sub + 3) / 4;
}

/* Build from signatures.  On success *blob receives a malloc'ed array of
 * *words 64-bit words holding the serialized structure.  extra = 0 builds
 * the minimal perfect hash function of the paper.  extra = e > 0 builds the
 * perfect, non-minimal variant: every leaf of m >= 2 keys maps its keys
 * injectively into m + e values, a bucket's output range is the sum of its
 * leaves' ranges, and the first Elias-Fano list holds the prefix sums of the
 * bucket ranges instead of the bucket sizes (a bucket's size is the one
 * whose range is the difference).  leaf + extra <= 32. */
int orc_build_fingerprints_e(const uint64_t* hi, const uint64_t* lo, uint64_t n, uint32_t leaf, uint32_t extra,
                             uint32_t bucket_size, int threads, uint64_t** blob, uint64_t* words) {
  if (leaf < 1 || leaf > 24 || bucket_size < 1 || bucket_size > 65535 || leaf + extra > 32) return ORC_E_INVALID;
  if (threads < 1) threads = 1;
  uint64_t nb = (n + bucket_size - 1) / bucket_size;
  int rc = ORC_E_NOMEM;

  /* Sec. 6.3: prefix sums of the bucket sizes, then group the keys. */
  uint64_t* bstart = calloc(nb + 2, sizeof(uint64_t));
  uint64_t* sorted = malloc((n + 1) * sizeof(uint64_t));
  uint64_t* fill = calloc(nb + 1, sizeof(uint64_t));
  uint64_t *cbase = NULL, *seeds = NULL, *sizes = NULL, *bits = NULL, *out = NULL, *rstart = NULL;
  orc_tables t;
  int have_tables = 0;
  if (!bstart || !sorted || !fill) goto done;
  for (uint64_t i = 0; i < n; i++) bstart[orc_bucket(hi[i], nb) + 1]++;
  uint64_t mmax = 0;
  for (uint64_t b = 0; b < nb; b++) {
    uint64_t m = bstart[b + 1];
    if (m > mmax) mmax = m;
    bstart[b + 1] += bstart[b];
  }
  for (uint64_t i = 0; i < n; i++) {
    uint64_t b = orc_bucket(hi[i], nb);
    sorted[bstart[b] + fill[b]++] = lo[i];
  }
  if ((rc = orc_tables_init(&t, leaf, extra, mmax < 2 ? 2 : mmax))) goto done;
  have_tables = 1;
  rc = ORC_E_NOMEM;
  /* prefix sums of the bucket output ranges (the bucket sizes when e = 0) */
  rstart = calloc(nb + 2, sizeof(uint64_t));
  if (!rstart) goto done;
  for (uint64_t b = 0; b < nb; b++) rstart[b + 1] = rstart[b] + t.rng[bstart[b + 1] - bstart[b]];
  uint64_t nrange = rstart[nb];

  /* Code slots: bucket b owns codes(m_b) consecutive slots. */
  cbase = calloc(nb + 1, sizeof(uint64_t));
  if (!cbase) goto done;
  for (uint64_t b = 0; b < nb; b++) {
    uint64_t m = bstart[b + 1] - bstart[b];
    cbase[b + 1] = cbase[b] + (m < 2 ? 0 : t.codes[m]);
  }
  uint64_t ncodes = cbase[nb];
  seeds = calloc(ncodes + 1, sizeof(uint64_t));
  sizes = calloc(ncodes + 1, sizeof(uint64_t));
  if (!seeds || !sizes) goto done;

  {
    orc_job jobs[256];
    pthread_t tid[256];
    if (threads > 256) threads = 256;
    uint64_t per = (nb + threads - 1) / (uint64_t)threads;
    int started[256] = {0};
    for (int k = 0; k < threads; k++) {
      jobs[k] = (orc_job){&t, sorted, bstart, cbase, seeds, sizes, 0, 0, 0};
      jobs[k].b0 = per * k < nb ? per * k : nb;
      jobs[k].b1 = per * (k + 1) < nb ? per * (k + 1) : nb;
    }
    if (threads == 1) {
      orc_worker(&jobs[0]);
    } else {
      for (int k = 0; k < threads; k++) {
        if (pthread_create(&tid[k], NULL, orc_worker, &jobs[k]) != 0)
          orc_worker(&jobs[k]);
        else
          started[k] = 1;
      }
      for (int k = 0; k < threads; k++)
        if (started[k]) pthread_join(tid[k], NULL);
    }
    rc = ORC_OK;
    for (int k = 0; k < threads; k++)
      if (jobs[k].rc && rc == ORC_OK) rc = jobs[k].rc;
    if (rc) goto done;
  }

  /* Sec. 6.2: per bucket, all fixed parts in preorder, then all unary parts.
   * A code for index i with parameter r is the low r bits of i (fixed part)
   * and i >> r zeros followed by a one (unary part). */
  uint64_t* off = calloc(nb + 1, sizeof(uint64_t));
  if (!off) {
    rc = ORC_E_NOMEM;
    goto done;
  }
  for (uint64_t b = 0; b < nb; b++) {
    uint64_t m = bstart[b + 1] - bstart[b];
    uint64_t len = m < 2 ? 0 : t.fbits[m];
    for (uint64_t c = cbase[b]; c < cbase[b + 1]; c++) len += (seeds[c] >> t.r[sizes[c]]) + 1;
    off[b + 1] = off[b] + len;
  }
  uint64_t T = off[nb];
  bits = calloc(orc_words(T) + 1, sizeof(uint64_t));
  if (!bits) {
    free(off);
    rc = ORC_E_NOMEM;
    goto done;
  }
  for (uint64_t b = 0; b < nb; b++) {
    uint64_t m = bstart[b + 1] - bstart[b];
    uint64_t fpos = off[b], upos = off[b] + (m < 2 ? 0 : t.fbits[m]);
    for (uint64_t c = cbase[b]; c < cbase[b + 1]; c++) {
      int r = t.r[sizes[c]];
      orc_put_bits(bits, fpos, seeds[c] & ((r == 64) ? ~0ULL : ((1ULL << r) - 1)), r);
      fpos += (uint64_t)r;
      upos += seeds[c] >> r;
      orc_put_bits(bits, upos, 1, 1);
      upos += 1;
    }
  }

  /* Sec. 6.3 / Sec. 7.4: double Elias-Fano of s_i and o_i - beta s_i (with
   * the range prefix sums in place of s_i in the non-minimal variant). */
  uint64_t beta = nrange ? (uint64_t)(((u128)T << 32) / nrange) : 0;
  uint64_t* xa = malloc((nb + 1) * sizeof(uint64_t));
  int64_t* z = malloc((nb + 1) * sizeof(int64_t));
  uint64_t* xb = malloc((nb + 1) * sizeof(uint64_t));
  if (!xa || !z || !xb) {
    free(off);
    free(xa);
    free(z);
    free(xb);
    rc = ORC_E_NOMEM;
    goto done;
  }
  int64_t da = 0, db = 0;
  for (uint64_t i = 0; i < nb; i++) {
    int64_t d = (int64_t)(rstart[i + 1] - rstart[i]);
    if (i == 0 || d < da) da = d;
  }
  for (uint64_t i = 0; i <= nb; i++) z[i] = (int64_t)off[i] - (int64_t)(((u128)rstart[i] * beta) >> 32);
  for (uint64_t i = 0; i < nb; i++) {
    int64_t d = z[i + 1] - z[i];
    if (i == 0 || d < db) db = d;
  }
  for (uint64_t i = 0; i <= nb; i++) {
    xa[i] = rstart[i] - (uint64_t)((int64_t)i * da);
    xb[i] = (uint64_t)(z[i] - (int64_t)i * db);
  }
  int la = orc_ef_width(xa[nb], nb + 1), lb = orc_ef_width(xb[nb], nb + 1);
  uint64_t ua = (xa[nb] >> la) + nb + 1, ub = (xb[nb] >> lb) + nb + 1;

  uint64_t h[ORC_HEADER_WORDS] = {0};
  h[0] = ORC_MAGIC;
  h[1] = n;
  h[2] = leaf | ((uint64_t)extra << 8);
  h[3] = bucket_size;
  h[4] = nb;
  h[5] = T;
  h[6] = mmax;
  h[7] = beta;
  h[8] = (uint64_t)da;
  h[9] = (uint64_t)db;
  h[10] = (uint64_t)la;
  h[11] = (uint64_t)lb;
  h[12] = ua;
  h[13] = ub;
  h[15] = ncodes;
  orc_layout L;
  orc_layout_of(h, &L);
  h[14] = L.total;
  out = calloc(L.total, sizeof(uint64_t));
  if (!out) {
    free(off);
    free(xa);
    free(z);
    free(xb);
    rc = ORC_E_NOMEM;
    goto done;
  }
  memcpy(out, h, sizeof(h));
  memcpy(out + L.tree, bits, orc_words(T) * sizeof(uint64_t));
  for (uint64_t i = 0; i <= nb; i++) {
    uint64_t rec = i * (uint64_t)(la + lb);
    orc_put_bits(out + L.lower, rec, xa[i] & ((1ULL << la) - 1), la);
    orc_put_bits(out + L.lower, rec + la, xb[i] & ((1ULL << lb) - 1), lb);
    orc_put_bits(out + L.upper_a, (xa[i] >> la) + i, 1, 1);
    orc_put_bits(out + L.upper_b, (xb[i] >> lb) + i, 1, 1);
  }
  uint16_t* subs = (uint16_t*)(out + L.subs);
  for (uint64_t k = 0; k < L.n_anchor; k++) {
    uint64_t i = k << ORC_INV_HI;
    out[L.anchors + 2 * k] = (xa[i] >> la) + i;
    out[L.anchors + 2 * k + 1] = (xb[i] >> lb) + i;
  }
  for (uint64_t j = 0; j < L.n_sub; j++) {
    uint64_t i = j << ORC_INV_LO, k = i >> ORC_INV_HI;
    uint64_t da_ = (xa[i] >> la) + i - out[L.anchors + 2 * k];
    uint64_t db_ = (xb[i] >> lb) + i - out[L.anchors + 2 * k + 1];
    subs[2 * j] = (uint16_t)(da_ < 0xFFFF ? da_ : 0xFFFF);
    subs[2 * j + 1] = (uint16_t)(db_ < 0xFFFF ? db_ : 0xFFFF);
  }
  free(off);
  free(xa);
  free(z);
  free(xb);
  *blob = out;
  *words = L.total;
  out = NULL;
  rc = ORC_OK;

done:
  if (have_tables) orc_tables_free(&t);
  free(bstart);
  free(sorted);
  free(fill);
  free(cbase);
  free(seeds);
  free(sizes);
  free(bits);
  free(out);
  free(rstart);
  return rc;
}

int orc_build_fingerprints(const uint64_t* hi, const uint64_t* lo, uint64_t n, uint32_t leaf,
                           uint32_t bucket_size, int threads, uint64_t** blob, uint64_t* words) {
  return orc_build_fingerprints_e(hi, lo, n, leaf, 0, bucket_size, threads, blob, words);
}

int orc_build_u64_e(const uint64_t* keys, uint64_t n, uint32_t leaf, uint32_t extra, uint32_t bucket_size,
                    int threads, uint64_t** blob, uint64_t* words) {
  uint64_t* hi = malloc((n + 1) * sizeof(uint64_t));
  uint64_t* lo = malloc((n + 1) * sizeof(uint64_t));
  if (!hi || !lo) {
    free(hi);
    free(lo);
    return ORC_E_NOMEM;
  }
  orc_fingerprint_u64(keys, n, hi, lo);
  int rc = orc_build_fingerprints_e(hi, lo, n, leaf, extra, bucket_size, threads, blob, words);
  free(hi);
  free(lo);
  return rc;
}

int orc_build_u64(const uint64_t* keys, uint64_t n, uint32_t leaf, uint32_t bucket_size, int threads,
                  uint64_t** blob, uint64_t* words) {
  uint64_t* hi = malloc((n + 1) * sizeof(uint64_t));
  uint64_t* lo = malloc((n + 1) * sizeof(uint64_t));
  if (!hi || !lo) {
    free(hi);
    free(lo);
    return ORC_E_NOMEM;
  }
  orc_fingerprint_u64(keys, n, hi, lo);
  int rc = orc_build_fingerprints(hi, lo, n, leaf, bucket_size, threads, blob, words);
  free(hi);
  free(lo);
  return rc;
}

int orc_build_bytes(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, uint32_t leaf,
                    uint32_t bucket_size, int threads, uint64_t** blob, uint64_t* words) {
  uint64_t* hi = malloc((n + 1) * sizeof(uint64_t));
  uint64_t* lo = malloc((n + 1) * sizeof(uint64_t));
  if (!hi || !lo) {
    free(hi);
    free(lo);
    return ORC_E_NOMEM;
  }
  orc_fingerprint_bytes(bytes, offsets, n, hi, lo);
  int rc = orc_build_fingerprints(hi, lo, n, leaf, bucket_size, threads, blob, words);
  free(hi);
  free(lo);
  return rc;
}

int orc_build_bytes_e(const uint8_t* bytes, const uint64_t* offsets, uint64_t n, uint32_t leaf, uint32_t extra,
                      uint32_t bucket_size, int threads, uint64_t** blob, uint64_t* words) {
  uint64_t* hi = malloc((n + 1) * sizeof(uint64_t));
  uint64_t* lo = malloc((n + 1) * sizeof(uint64_t));
  if (!hi || !lo) {
    free(hi);
    free(lo);
    return ORC_E_NOMEM;
  }
  orc_fingerprint_bytes(bytes, offsets, n, hi, lo);
  int rc = orc_build_fingerprints_e(hi, lo, n, leaf, extra, bucket_size, threads, blob, words);
  free(hi);
  free(lo);
  return rc;
}

void orc_free(void* p) { free(p); }

/* ------------------------------------------------------------------ */
/* Decoding (Sec. 7.4 select, Sec. 6.2 tree walk) and lookup (Sec. 4). */
/* ------------------------------------------------------------------ */
/* Position of the one of rank `rank` (0-based) in an upper-bits array,
 * starting from the 16-bit inventory entry at or before it (entries that
 * did not fit in 16 bits hold 0xFFFF and are passed over) and counting ones
 * word by word. */
static uint64_t orc_select(const uint64_t* blob, const orc_layout* L, int list, uint64_t rank) {
  const uint64_t* up = blob + (list ? L->upper_b : L->upper_a);
  const uint16_t* subs = (const uint16_t*)(blob + L->subs);
  uint64_t k = rank >> ORC_INV_HI;
  uint64_t j = rank >> ORC_INV_LO;
  uint64_t first_j = k << (ORC_INV_HI - ORC_INV_LO);
  /* the entry of the anchor itself is always 0, so this stops there */
  while (j > first_j && subs[2 * j + list] == 0xFFFF) j--;
  uint64_t pos = blob[L->anchors + 2 * k + list] + subs[2 * j + list];
  uint64_t need = rank - (j << ORC_INV_LO); /* further ones after the one at pos */
  uint64_t w = pos >> 6;
  uint64_t word = up[w] & (~0ULL << (pos & 63));
  for (;;) {
    uint64_t c = (uint64_t)__builtin_popcountll(word);
    if (need < c) break;
    need -= c;
    word = up[++w];
  }
  for (uint64_t s = 0; s < need; s++) word &= word - 1;
  return w * 64 + (uint64_t)__builtin_ctzll(word);
}

/* Element i of list 0 (rescaled prefix sums) or 1 (rescaled offsets). */
static uint64_t orc_ef_get(const uint64_t* blob, const orc_layout* L, int list, uint64_t i) {
  uint64_t la = blob[10], lb = blob[11];
  uint64_t width = list ? lb : la;
  uint64_t lowpos = i * (la + lb) + (list ? la : 0);
  uint64_t low = orc_get_bits(blob + L->lower, lowpos, (int)width);
  uint64_t high = orc_select(blob, L, list, i) - i;
  return (high << width) | low;
}

/* s_i and o_i of bucket i, undoing the rescaling by the minimum deltas and
 * by beta. */
int orc_bucket_info(const uint64_t* blob, uint64_t i, uint64_t* s, uint64_t* o) {
  orc_layout L;
  orc_layout_of(blob, &L);
  if (i > blob[4]) return ORC_E_INVALID;
  int64_t da = (int64_t)blob[8], db = (int64_t)blob[9];
  uint64_t sv = orc_ef_get(blob, &L, 0, i) + (uint64_t)((int64_t)i * da);
  int64_t zv = (int64_t)orc_ef_get(blob, &L, 1, i) + (int64_t)i * db;
  *s = sv;
  *o = (uint64_t)(zv + (int64_t)(((u128)sv * blob[7]) >> 32));
  return ORC_OK;
}

static uint64_t orc_next_unary(const uint64_t* tree, uint64_t* upos) {
  uint64_t q = 0;
  while (!orc_get_bit(tree, *upos)) {
    q++;
    (*upos)++;
  }
  (*upos)++;
  return q;
}

/* Indices of bucket b in preorder, read back from the bit array by walking
 * the fixed and unary parts in step (no skipping). */
int orc_decode_bucket(const uint64_t* blob, uint64_t b, uint64_t* seeds, uint64_t cap, uint64_t* count) {
  orc_layout L;
  orc_layout_of(blob, &L);
  if (b >= blob[4]) return ORC_E_INVALID;
  uint64_t s0, s1, o0, o1;
  orc_bucket_info(blob, b, &s0, &o0);
  orc_bucket_info(blob, b + 1, &s1, &o1);
  orc_tables t;
  int rct = orc_tables_init(&t, (uint32_t)(blob[2] & 0xFF), (uint32_t)((blob[2] >> 8) & 0xFF), blob[6] < 2 ? 2 : blob[6]);
  if (rct) return rct;
  uint64_t m = orc_size_of_range(&t, s1 - s0);
  if (m == UINT64_MAX) {
    orc_tables_free(&t);
    return ORC_E_INVALID;
  }
  /* preorder list of node sizes, expanded with an explicit stack */
  uint64_t* stack = malloc((64 * ORC_MAX_FANOUT + 1) * sizeof(uint64_t));
  uint64_t sp = 0, k = 0;
  const uint64_t* tree = blob + L.tree;
  uint64_t fpos = o0, upos = o0 + (m < 2 ? 0 : t.fbits[m]);
  if (m >= 2) stack[sp++] = m;
  while (sp) {
    uint64_t sz = stack[--sp];
    if (sz < 2) continue;
    int r = t.r[sz];
    uint64_t low = orc_get_bits(tree, fpos, r);
    fpos += (uint64_t)r;
    uint64_t q = orc_next_unary(tree, &upos);
    if (k < cap) seeds[k] = (q << r) | low;
    k++;
    if (sz > t.leaf) {
      uint64_t parts[ORC_MAX_FANOUT], u;
      int f = orc_strategy(t.leaf, sz, &u, parts, ORC_MAX_FANOUT);
      for (int j = f - 1; j >= 0; j--) stack[sp++] = parts[j];
    }
  }
  *count = k;
  free(stack);
  /* the code must end exactly where the next bucket's begins (checked
   * before the tables it reads are released) */
  const int ok = upos == o1 && fpos == o0 + (m < 2 ? 0 : t.fbits[m]);
  orc_tables_free(&t);
  return ok ? ORC_OK : ORC_E_INVALID;
}

typedef struct {
  uint64_t n, leaf, nb;
  orc_layout L;
  orc_tables t;
} orc_reader;

static int orc_reader_init(orc_reader* rd, const uint64_t* blob) {
  if (blob[0] != ORC_MAGIC) return ORC_E_INVALID;
  rd->n = blob[1];
  rd->leaf = blob[2] & 0xFF;
  rd->nb = blob[4];
  orc_layout_of(blob, &rd->L);
  return orc_tables_init(&rd->t, (uint32_t)rd->leaf, (uint32_t)((blob[2] >> 8) & 0xFF), blob[6] < 2 ? 2 : blob[6]);
}

/* Sec. 4: descend from the root with the split indices; every move to
 * child j leaves the j earlier siblings (and their keys) to the left, whose
 * fixed bits are skipped with the table and whose unary codes are skipped by
 * counting ones (Sec. 6.2); at the leaf add the bijection's value.  In the
 * non-minimal variant the siblings left behind count with their output
 * ranges and the leaf's value lies in [0, m + e). */
static uint64_t orc_lookup_one(const orc_reader* rd, const uint64_t* blob, uint64_t hi, uint64_t lo) {
  if (rd->nb == 0) return 0;
  uint64_t b = orc_bucket(hi, rd->nb);
  uint64_t s0, s1, o0, o1;
  orc_bucket_info(blob, b, &s0, &o0);
  orc_bucket_info(blob, b + 1, &s1, &o1);
  uint64_t m = orc_size_of_range(&rd->t, s1 - s0);
  if (m == UINT64_MAX) return s0;  /* not a structure this reader wrote */
  const uint64_t* tree = blob + rd->L.tree;
  uint64_t fpos = o0, upos = o0 + (m < 2 ? 0 : rd->t.fbits[m]), c = 0;
  uint32_t depth = 0;
  for (;;) {
    if (m <= 1) return s0 + c;
    int r = rd->t.r[m];
    uint64_t low = orc_get_bits(tree, fpos, r);
    fpos += (uint64_t)r;
    uint64_t q = orc_next_unary(tree, &upos);
    uint64_t seed = (q << r) | low;
    if (m <= rd->leaf) return s0 + c + orc_phi(lo, depth, seed, m + rd->t.extra);
    uint64_t v = orc_phi(lo, depth, seed, m);
    uint64_t parts[ORC_MAX_FANOUT], u;
    int f = orc_strategy((uint32_t)rd->leaf, m, &u, parts, ORC_MAX_FANOUT);
    uint64_t lim = 0;
    int p = 0;
    for (;;) {
      lim += parts[p];
      if (v < lim || p == f - 1) break;
      p++;
    }
    for (int j = 0; j < p; j++) {
      fpos += rd->t.fbits[parts[j]];
      for (uint64_t skip = rd->t.codes[parts[j]]; skip; skip--) orc_next_unary(tree, &upos);
      c += rd->t.rng[parts[j]];
    }
    m = parts[p];
    depth++;
  }
}

int orc_lookup_fingerprints(const uint64_t* blob, const uint64_t* hi, const uint64_t* lo, uint64_t q,
                            uint64_t* out) {
  orc_reader rd;
  int rc = orc_reader_init(&rd, blob);
  if (rc) return rc;
  for (uint64_t i = 0; i < q; i++) out[i] = orc_lookup_one(&rd, blob, hi[i], lo[i]);
  orc_tables_free(&rd.t);
  return ORC_OK;
}

int orc_lookup_u64(const uint64_t* blob, const uint64_t* keys, uint64_t q, uint64_t* out) {
  orc_reader rd;
  int rc = orc_reader_init(&rd, blob);
  if (rc) return rc;
  for (uint64_t i = 0; i < q; i++) {
    uint64_t hi = orc_mix64(keys[i] ^ ORC_FP_HI), lo = orc_mix64(keys[i] ^ ORC_FP_LO);
    out[i] = orc_lookup_one(&rd, blob, hi, lo);
  }
  orc_tables_free(&rd.t);
  return ORC_OK;
}

int orc_lookup_bytes(const uint64_t* blob, const uint8_t* bytes, const uint64_t* offsets, uint64_t q,
                     uint64_t* out) {
  orc_reader rd;
  int rc = orc_reader_init(&rd, blob);
  if (rc) return rc;
  for (uint64_t i = 0; i < q; i++) {
    uint64_t hi, lo;
    orc_fingerprint_one_bytes(bytes + offsets[i], offsets[i + 1] - offsets[i], &hi, &lo);
    out[i] = orc_lookup_one(&rd, blob, hi, lo);
  }
  orc_tables_free(&rd.t);
  return ORC_OK;
}

/* Plain linear select (no inventory), for checking the inventory. */
uint64_t orc_select_linear(const uint64_t* blob, int list, uint64_t rank) {
  orc_layout L;
  orc_layout_of(blob, &L);
  const uint64_t* up = blob + (list ? L.upper_b : L.upper_a);
  uint64_t len = list ? blob[13] : blob[12];
  uint64_t seen = 0;
  for (uint64_t p = 0; p < len; p++)
    if (orc_get_bit(up, p)) {
      if (seen == rank) return p;
      seen++;
    }
  return ~0ULL;
}

uint64_t orc_select_inventory(const uint64_t* blob, int list, uint64_t rank) {
  orc_layout L;
  orc_layout_of(blob, &L);
  return orc_select(blob, &L, list, rank);
}

/* Section word offsets, for tests that look inside the structure. */
void orc_layout_words(const uint64_t* blob, uint64_t* out7) {
  orc_layout L;
  orc_layout_of(blob, &L);
  out7[0] = L.tree;
  out7[1] = L.lower;
  out7[2] = L.upper_a;
  out7[3] = L.upper_b;
  out7[4] = L.anchors;
  out7[5] = L.subs;
  out7[6] = L.total;
}
