// Host-side tables: splitting strategy (Sec. 5.4), Golomb-Rice parameters
// (Sec. 5.4 Eq. gr, Sec. 7.2) and the subtree skip information of Sec. 6.2.
#include <cmath>
#include <cstdio>

#include "common.h"

namespace rs {

Layout layout_of(const uint64_t* h) {
  Layout L;
  const uint64_t nb = h[H_NB];
  L.n_anchor = (nb >> kInvHi) + 1;
  L.n_sub = (nb >> kInvLo) + 1;
  L.tree = kHeaderWords;
  L.lower = L.tree + words_of_bits(h[H_TBITS]);
  L.upper_a = L.lower + words_of_bits((nb + 1) * (h[H_LOW_A] + h[H_LOW_B]));
  L.upper_b = L.upper_a + words_of_bits(h[H_UP_A]);
  L.anchors = L.upper_b + words_of_bits(h[H_UP_B]);
  L.subs = L.anchors + 2 * L.n_anchor;
  L.total = L.subs + (2 * L.n_sub * sizeof(uint16_t) + 7) / 8;
  return L;
}

// Sec. 5.4: s = max(2, ceil(0.35 l + 0.5)) leaves are aggregated first, then
// t = ceil(0.21 l + 0.9) (l >= 7; 2 below) such groups; the decimal
// coefficients are applied as exact fractions (7/20, 1/2, 21/100, 9/10).
Strategy make_strategy(uint32_t leaf) {
  const uint64_t l = leaf;
  uint64_t s = (7 * l + 10 + 19) / 20;
  if (s < 2) s = 2;
  const uint64_t t = l >= 7 ? (21 * l + 90 + 99) / 100 : 2;
  return Strategy{leaf, s * l, s * t * l};
}

Shape shape_of(const Strategy& st, uint64_t m) {
  if (m <= st.leaf) return Shape{0, 0, 0};
  if (m > st.upper) {
    // fanout 2; the left part is floor(m/2) rounded up to a multiple of s*t*l
    const uint64_t left = (m / 2 + st.upper - 1) / st.upper * st.upper;
    return Shape{2, left, m - left};
  }
  const uint64_t unit = m <= st.lower ? st.leaf : st.lower;
  const uint64_t fanout = (m + unit - 1) / unit;
  return Shape{static_cast<uint32_t>(fanout), unit, m - unit * (fanout - 1)};
}

static int floor_log2(uint64_t x) { return x ? 63 - __builtin_clzll(x) : 0; }

// ln of the probability that one trial succeeds at a node of m keys:
// m!/m^m for a leaf (Sec. 5.2); for a split Eq. probsplit, i.e. that times
// k^k/k! for every part k (Sec. 5.1).  With leaf range extra e a leaf trial
// succeeds when its m values are distinct in [0, R), R = m + e:
// R! / ((R - m)! R^m) (m!/m^m for e = 0).
static double log_trial_success(const Strategy& st, uint64_t m) {
  const double dm = static_cast<double>(m);
  const Shape sh = shape_of(st, m);
  if (sh.fanout == 0) {
    const double dr = static_cast<double>(m + st.extra);
    return std::lgamma(dr + 1.0) - std::lgamma(dr - dm + 1.0) - dm * std::log(dr);
  }
  double v = std::lgamma(dm + 1.0) - dm * std::log(dm);
  auto term = [](uint64_t k) {
    const double dk = static_cast<double>(k);
    return dk * std::log(dk) - std::lgamma(dk + 1.0);
  };
  v += static_cast<double>(sh.fanout - 1) * term(sh.unit);
  v += term(sh.last);
  return v;
}

int golomb_rice_param(const Strategy& st, uint64_t m) {
  if (m < 2) return 0;
  if (m < 65536) {
    // Eq. gr: r = max(0, ceil(lg(-lg(phi) / lg(1 - p))))
    const double p = std::exp(log_trial_success(st, m));
    const double phi = 0.5 * (1.0 + std::sqrt(5.0));
    const double x = std::log2(-std::log(phi) / std::log1p(-p));
    const double c = std::ceil(x);
    return c > 0.0 ? static_cast<int>(c) : 0;
  }
  // Sec. 7.2 integer approximation for large nodes (">>" as a right shift)
  const Shape sh = shape_of(st, m);
  int64_t v = static_cast<int64_t>(((sh.fanout - 1) * 5ull) >> 1);
  v += static_cast<int64_t>(sh.fanout - 1) * floor_log2(sh.unit + (sh.unit >> 1));
  v += floor_log2(sh.last + (sh.last >> 1));
  v -= floor_log2(m);
  return v > 0 ? static_cast<int>(v >> 1) : 0;
}

int build_tables(uint32_t leaf, uint32_t extra, uint64_t mmax, Tables* T, std::string* err) {
  Strategy st = make_strategy(leaf);
  st.extra = extra;
  if (mmax < 2) mmax = 2;
  T->mmax = mmax;
  T->r.assign(mmax + 1, 0);
  T->fixed_bits.assign(mmax + 1, 0);
  T->codes.assign(mmax + 1, 0);
  T->expected_trials.assign(mmax + 1, 0);
  T->range.assign(mmax + 1, 0);
  // the search tables, then the lookup records (two words per size)
  T->device_words.assign((kTableWords + 2) * (mmax + 1), 0);
  LookupRecord* rec = reinterpret_cast<LookupRecord*>(T->device_words.data() + kTableWords * (mmax + 1));
  // sizes 0 and 1: no code, output range m
  T->range[1] = 1;
  T->device_words[kTableWords * 1 + 3] = uint64_t(1) << 32;
  for (uint64_t m = 2; m <= mmax; m++) {
    const Shape sh = shape_of(st, m);
    const int r = golomb_rice_param(st, m);
    uint64_t fb = static_cast<uint64_t>(r), nc = 1;
    if (sh.fanout) {
      fb += (sh.fanout - 1) * T->fixed_bits[sh.unit] + T->fixed_bits[sh.last];
      nc += (sh.fanout - 1) * T->codes[sh.unit] + T->codes[sh.last];
    }
    T->r[m] = static_cast<uint8_t>(r);
    T->fixed_bits[m] = fb;
    T->codes[m] = nc;
    T->range[m] = sh.fanout ? (sh.fanout - 1) * T->range[sh.unit] + T->range[sh.last] : m + extra;
    // a bucket's size is read back from its output range: the range must
    // grow strictly with the size (checked for every size)
    if (T->range[m] <= T->range[m - 1] || T->range[m] >= (1ull << 32)) {
      if (err) *err = "subtree output ranges do not grow with the node size";
      return RECSPLIT_E_INVALID;
    }
    const double et = std::exp(-log_trial_success(st, m));
    T->expected_trials[m] = et > 1e18 ? ~0ull : static_cast<uint64_t>(std::ceil(et));
    if (fb >= (1ull << 32) || nc >= (1ull << 32) || r >= 32 || sh.unit >= (1ull << 32)) {
      if (err) *err = "node size too large for the device tables";
      return RECSPLIT_E_INVALID;
    }
    T->device_words[kTableWords * m] = fb | (nc << 32);
    T->device_words[kTableWords * m + 1] =
        sh.unit | (static_cast<uint64_t>(sh.fanout) << 32) | (static_cast<uint64_t>(r) << 40);
    T->device_words[kTableWords * m + 2] = T->expected_trials[m];
    // word 3, lower half: M = ceil(2^32 / unit), with which floor(v * M / 2^32)
    // = floor(v / unit) for every v < m when (m - 1) * (M * unit - 2^32) < 2^32
    // (always for m < 2^16); 0 where that fails, and the lookup divides
    uint64_t magic = 0;
    if (sh.unit >= 2) {
      const uint64_t M = ((1ull << 32) + sh.unit - 1) / sh.unit;
      if ((m - 1) * (M * sh.unit - (1ull << 32)) < (1ull << 32)) magic = M;
    }
    T->device_words[kTableWords * m + 3] = magic | (T->range[m] << 32);
    const uint64_t unit_codes = sh.fanout ? T->codes[sh.unit] : 0;
    if (unit_codes >= (1ull << kLookupCodeBits) || sh.fanout >= 16) {
      if (err) *err = "node size too large for the lookup records";
      return RECSPLIT_E_INVALID;
    }
    rec[m].unit = static_cast<uint32_t>(sh.unit);
    rec[m].magic = static_cast<uint32_t>(magic);
    rec[m].fixed = static_cast<uint32_t>(sh.fanout ? T->fixed_bits[sh.unit] : 0);
    rec[m].info = static_cast<uint32_t>(unit_codes) | (static_cast<uint32_t>(r) << kLookupCodeBits) |
                  (sh.fanout << 28);
  }
  return RECSPLIT_OK;
}

}  // namespace rs

extern "C" int recsplit_golomb_rice_params_extra(uint32_t leaf_size, uint32_t leaf_extra, uint64_t m_hi,
                                                 uint8_t* out) {
  if (leaf_size < 1 || leaf_size > rs::kMaxLeaf || leaf_size + leaf_extra > 32 || !out) return RECSPLIT_E_INVALID;
  rs::Strategy st = rs::make_strategy(leaf_size);
  st.extra = leaf_extra;
  for (uint64_t m = 0; m <= m_hi; m++) out[m] = static_cast<uint8_t>(rs::golomb_rice_param(st, m));
  return RECSPLIT_OK;
}

extern "C" int recsplit_golomb_rice_params(uint32_t leaf_size, uint64_t m_hi, uint8_t* out) {
  if (leaf_size < 1 || leaf_size > rs::kMaxLeaf || !out) return RECSPLIT_E_INVALID;
  const rs::Strategy st = rs::make_strategy(leaf_size);
  for (uint64_t m = 0; m <= m_hi; m++) out[m] = static_cast<uint8_t>(rs::golomb_rice_param(st, m));
  return RECSPLIT_OK;
}
