// Host-side check of a serialized structure before it is loaded
// (recsplit_deserialize).  A lookup reads the bucket's prefix sum and bit
// offset from the double Elias-Fano lists (Sec. 6.3, Sec. 7.4) through their
// inventories, then walks the bucket's Golomb-Rice codes (Sec. 6.2), finding
// unary codes by scanning for one bits.  The device code trusts what it reads,
// so every part of the structure that steers those reads is checked here:
//  - each upper-bits array holds exactly N + 1 one bits;
//  - the u64 anchors and u16 offsets of the inventories are the positions the
//    lists' one bits give (the writer's rule, 0xFFFF where an offset does not
//    fit in 16 bits; 0xFFFF, which makes select use an earlier entry, is also
//    accepted elsewhere except at the first entry of an anchor's block);
//  - the decoded prefix sums start at 0, never decrease, end at the output
//    range, and every bucket's size (with a leaf range extra, the size whose
//    output range is the bucket's) is at most the header's largest bucket;
//  - the decoded bit offsets start at 0, never decrease and end at the tree
//    size T;
//  - the code of a bucket of m >= 2 keys spans at least its fixed bits plus
//    one bit per code, under 2^32 bits, and its unary part holds exactly as
//    many one bits as its tree has codes, the last bit being one; a bucket of
//    0 or 1 keys has no code.
#include <cstring>
#include <string>
#include <vector>

#include "common.h"

namespace rs {
namespace {

uint64_t get_bits(const uint64_t* a, uint64_t pos, uint32_t width) {
  if (width == 0) return 0;
  const uint64_t w = pos >> 6;
  const uint32_t o = static_cast<uint32_t>(pos & 63);
  uint64_t v = a[w] >> o;
  if (o + width > 64) v |= a[w + 1] << (64 - o);
  return width == 64 ? v : (v & ((1ull << width) - 1));
}

// One bits in [from, to) of a bit array.
uint64_t ones_between(const uint64_t* a, uint64_t from, uint64_t to) {
  if (from >= to) return 0;
  uint64_t c = 0;
  const uint64_t w0 = from >> 6, w1 = (to - 1) >> 6;
  for (uint64_t w = w0; w <= w1; w++) {
    uint64_t word = a[w];
    if (w == w0) word &= ~0ull << (from & 63);
    if (w == w1 && (to & 63)) word &= ~0ull >> (64 - (to & 63));
    c += static_cast<uint64_t>(__builtin_popcountll(word));
  }
  return c;
}

// Positions of the one bits of an upper-bits array of `bits` bits, which must
// hold exactly `count` of them.
bool one_positions(const uint64_t* a, uint64_t bits, uint64_t count, std::vector<uint64_t>* pos) {
  pos->clear();
  pos->reserve(count);
  const uint64_t words = words_of_bits(bits);
  for (uint64_t w = 0; w < words; w++) {
    uint64_t word = a[w];
    if (w + 1 == words && (bits & 63)) word &= ~0ull >> (64 - (bits & 63));
    while (word) {
      if (pos->size() == count) return false;
      pos->push_back((w << 6) + static_cast<uint64_t>(__builtin_ctzll(word)));
      word &= word - 1;
    }
  }
  return pos->size() == count;
}

int bad(std::string* err, const char* what) {
  *err = std::string("structure check failed: ") + what;
  return RECSPLIT_E_INVALID;
}

}  // namespace

// Decodes both lists of the structure `w` (header H, layout L) into s (prefix
// sums of the bucket output ranges) and o (bit offsets), N + 1 entries each,
// checking the inventories and the orders.
int check_lists(const uint64_t* w, const uint64_t* H, const Layout& L, std::vector<uint64_t>* s,
                std::vector<uint64_t>* o, std::string* err) {
  const uint64_t nb = H[H_NB];
  const uint32_t la = static_cast<uint32_t>(H[H_LOW_A]), lb = static_cast<uint32_t>(H[H_LOW_B]);
  const uint64_t* lower = w + L.lower;
  const uint16_t* subs = reinterpret_cast<const uint16_t*>(w + L.subs);
  std::vector<uint64_t> p[2];
  if (!one_positions(w + L.upper_a, H[H_UP_A], nb + 1, &p[0]) || !one_positions(w + L.upper_b, H[H_UP_B], nb + 1, &p[1]))
    return bad(err, "an upper-bits array does not hold one bit per bucket boundary");
  for (int list = 0; list < 2; list++) {
    const std::vector<uint64_t>& q = p[list];
    for (uint64_t k = 0; k < L.n_anchor; k++)
      if (w[L.anchors + 2 * k + list] != q[k << kInvHi]) return bad(err, "an inventory anchor is wrong");
    for (uint64_t j = 0; j < L.n_sub; j++) {
      // 0xFFFF sends select to an earlier entry of the same anchor block, so
      // it is acceptable anywhere but at the block's first entry
      const bool block_start = (j & ((1u << (kInvHi - kInvLo)) - 1)) == 0;
      const uint64_t d = q[j << kInvLo] - q[(j >> (kInvHi - kInvLo)) << kInvHi];
      const uint16_t e = subs[2 * j + list];
      if (e != (d < 0xFFFF ? d : 0xFFFF) && (e != 0xFFFF || block_start))
        return bad(err, "an inventory offset is wrong");
    }
  }
  s->resize(nb + 1);
  o->resize(nb + 1);
  const int64_t da = static_cast<int64_t>(H[H_DELTA_A]), db = static_cast<int64_t>(H[H_DELTA_B]);
  for (uint64_t i = 0; i <= nb; i++) {
    const uint64_t rec = i * (la + lb);
    const uint64_t xa = ((p[0][i] - i) << la) | get_bits(lower, rec, la);
    const uint64_t xb = ((p[1][i] - i) << lb) | get_bits(lower, rec + la, lb);
    const uint64_t si = xa + static_cast<uint64_t>(static_cast<int64_t>(i) * da);
    const uint64_t bs = static_cast<uint64_t>((static_cast<unsigned __int128>(si) * H[H_BETA]) >> 32);
    (*s)[i] = si;
    (*o)[i] = static_cast<uint64_t>(static_cast<int64_t>(xb) + static_cast<int64_t>(i) * db) + bs;
    if (i && ((*s)[i] < (*s)[i - 1] || (*o)[i] < (*o)[i - 1]))
      return bad(err, "the prefix sums or bit offsets decrease");
  }
  if ((*s)[0] != 0 || (*o)[0] != 0) return bad(err, "the lists do not start at 0");
  if ((*o)[nb] != H[H_TBITS]) return bad(err, "the bit offsets do not end at the tree size");
  return RECSPLIT_OK;
}

// Bucket sizes from the output ranges s[i + 1] - s[i] (the ranges themselves
// when the tables have no leaf range extra), the codes of every bucket, and
// the number of codes.
int check_codes(const uint64_t* w, const uint64_t* H, const Layout& L, const Tables& T, uint32_t extra,
                const std::vector<uint64_t>& s, const std::vector<uint64_t>& o, std::string* err) {
  const uint64_t nb = H[H_NB];
  const uint64_t* tree = w + L.tree;
  uint64_t codes = 0;
  for (uint64_t i = 0; i < nb; i++) {
    const uint64_t R = s[i + 1] - s[i];
    uint64_t m = R;
    if (extra) {
      // ranges grow strictly with the size: binary search for the size
      uint64_t a = 0, b = T.mmax;
      while (a < b) {
        const uint64_t mid = (a + b + 1) >> 1;
        if (T.range[mid] <= R) a = mid; else b = mid - 1;
      }
      if (T.range[a] != R) return bad(err, "a bucket's output range belongs to no size");
      m = a;
    }
    if (m > T.mmax || m > H[H_MMAX]) return bad(err, "a bucket is larger than the header's largest bucket");
    const uint64_t len = o[i + 1] - o[i];
    if (m < 2) {
      if (len) return bad(err, "a bucket of fewer than two keys has a code");
      continue;
    }
    const uint64_t F = T.fixed_bits[m], C = T.codes[m];
    if (len < F + C || len >= (1ull << 32) - 64) return bad(err, "a bucket's code has the wrong length");
    if (ones_between(tree, o[i] + F, o[i + 1]) != C || !((tree[(o[i + 1] - 1) >> 6] >> ((o[i + 1] - 1) & 63)) & 1))
      return bad(err, "a bucket's unary codes do not match its tree");
    codes += C;
  }
  if (codes != H[H_CODES]) return bad(err, "the number of codes does not match the header");
  return RECSPLIT_OK;
}

}  // namespace rs
