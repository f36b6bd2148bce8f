// Device-side arithmetic of the structure: mixer, signatures, the hash family
// used by the searches, bit-array access and Elias-Fano select.
#pragma once

#include <cstdint>

#include "common.h"

namespace rs {

constexpr uint64_t kWeyl = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kMixA = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kMixB = 0x94D049BB133111EBull;
constexpr uint64_t kSigHi = 0x6A09E667F3BCC909ull;
constexpr uint64_t kSigLo = 0xBB67AE8584CAA73Bull;

// z >> S (0 < S < 32) for the signature mixer: the low word is a funnel shift
// (integer ALU pipe), the high word the multiply-high floor(hi * 2^(32-S) /
// 2^32), which issues to the multiply-add pipe.  The kernels that hash keys
// are bound by the ALU pipe (ncu, 10^6 string lookups: ALU pipe 75% busy,
// multiply-add pipe 21%), so this moves one instruction of every shift off
// it; measured on 10^8 string lookups: 3.78 -> 3.61 ms.  The same form in
// the search hash (family_top32) made the searches 3-6% slower: their
// multiply-add pipe already carries the hash's 64-bit multiplies.
template <int S>
__device__ __forceinline__ uint64_t shr_mix(uint64_t z) {
  const uint32_t lo = static_cast<uint32_t>(z), hi = static_cast<uint32_t>(z >> 32);
  uint32_t h;
  asm volatile("mul.hi.u32 %0, %1, %2;" : "=r"(h) : "r"(hi), "r"(1u << (32 - S)));
  return (uint64_t(h) << 32) | __funnelshift_r(lo, hi, S);
}

// splitmix64 finalizer (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
#ifdef __CUDA_ARCH__
  z = (z ^ shr_mix<30>(z)) * kMixA;
  z = (z ^ shr_mix<27>(z)) * kMixB;
  return z ^ shr_mix<31>(z);
#else
  z = (z ^ (z >> 30)) * kMixA;
  z = (z ^ (z >> 27)) * kMixB;
  return z ^ (z >> 31);
#endif
}

// ---------------------------------------------------------------- signatures
// Sec. 6.1: 128-bit signature of a 64-bit key, one mixer per half.
__device__ __forceinline__ void signature_u64(uint64_t key, uint64_t& hi, uint64_t& lo) {
  hi = mix64(key ^ kSigHi);
  lo = mix64(key ^ kSigLo);
}

// Signature of a byte string: 8-byte little-endian words (zero padded)
// absorbed by two mixer chains, the second on the word with its halves
// swapped, then the length folded into both.  The string is read with
// aligned 4-byte loads of the words that hold at least one of its bytes (no
// load leaves the page that holds the string); each 8-byte word is two funnel
// shifts of three consecutive loaded words.  Every 8-byte word but the last
// lies wholly inside the string, and so do the three 4-byte words it is cut
// from (the last of them holds the word's byte 8, which the string has), so
// those words are read without a bound or a mask; only the last 8-byte word
// (1 to 8 bytes) checks which loads the string covers and masks its tail.
__device__ __forceinline__ void absorb(uint64_t& a, uint64_t& c, uint64_t word) {
  a = mix64(a ^ word);
  c = mix64(c ^ ((word >> 32) | (word << 32)));
}

__device__ __forceinline__ void signature_bytes(const uint8_t* p, uint64_t len, uint64_t& hi, uint64_t& lo) {
  uint64_t a = kSigHi, c = kSigLo;
  if (len) {
    const uintptr_t addr = reinterpret_cast<uintptr_t>(p);
    const uint32_t* w = reinterpret_cast<const uint32_t*>(addr & ~uintptr_t(3));
    const uint32_t sh = static_cast<uint32_t>(addr & 3) * 8;
    const uint64_t nt = ((addr + len - 1) >> 2) - (addr >> 2) + 1;  // 4-byte words touched
    const uint64_t full = (len - 1) >> 3;                            // 8-byte words before the last
    uint32_t w0 = __ldg(w);
    // 32-bit trip counts (the outer loop runs more than once only for strings
    // of 32 GiB or more)
    for (uint64_t left = full; left;) {
      const uint32_t step = left < 0xFFFFFFFFull ? static_cast<uint32_t>(left) : 0xFFFFFFFFu;
      left -= step;
      for (uint32_t i = 0; i < step; i++) {
        const uint32_t w1 = __ldg(w + 1), w2 = __ldg(w + 2);
        w += 2;
        absorb(a, c, (uint64_t(__funnelshift_r(w1, w2, sh)) << 32) | __funnelshift_r(w0, w1, sh));
        w0 = w2;
      }
    }
    // the last 8-byte word: words 2 full + 1 and 2 full + 2 of the span,
    // each only where it holds a byte of the string
    const uint64_t j = 2 * full + 1;
    const uint32_t w1 = j < nt ? __ldg(w + 1) : 0u;
    const uint32_t w2 = j + 1 < nt ? __ldg(w + 2) : 0u;
    const uint32_t keep = static_cast<uint32_t>(len - 8 * full) * 8;  // 8 .. 64 bits of the word in the string
    const uint64_t word = ((uint64_t(__funnelshift_r(w1, w2, sh)) << 32) | __funnelshift_r(w0, w1, sh)) &
                          (~0ull >> (64 - keep));
    absorb(a, c, word);
  }
  hi = mix64(a + len);
  lo = mix64(c + len);
}

// Sec. 4 / 6.1: bucket by fixed-point inversion of the upper half.
__device__ __forceinline__ uint64_t bucket_of(uint64_t hi, uint64_t nb) { return __umul64hi(hi, nb); }

// ---------------------------------------------------------------- hash family
// Function i at depth d acts on the lower half x: z = x ^ K with
// K = (i * 64 + d) * W (W the Weyl constant), then the two xorshift-multiply
// rounds of the splitmix64 finalizer, keeping the top 32 bits;
// phi^m = floor(top32 * m / 2^32).  The searches keep, per key, the value
// x ^ (x >> 30) and, per function, K ^ (K >> 30): the first xorshift
// distributes over the xor, so it costs nothing per evaluation.
__host__ __device__ __forceinline__ uint64_t family_key(uint64_t index, uint32_t depth) {
  const uint64_t k = ((index << 6) | depth) * kWeyl;
  return k ^ (k >> 30);
}

__host__ __device__ __forceinline__ uint64_t pre_key(uint64_t x) { return x ^ (x >> 30); }

// Top 32 bits of the family's hash from the pre-shifted forms of x and K.
__device__ __forceinline__ uint32_t family_top32(uint64_t xpre, uint64_t kpre) {
  uint64_t z = (xpre ^ kpre) * kMixA;
  z ^= z >> 27;
  const uint32_t zl = static_cast<uint32_t>(z), zh = static_cast<uint32_t>(z >> 32);
  // high word of the low 64 bits of z * kMixB
  return __umulhi(zl, static_cast<uint32_t>(kMixB)) + zl * static_cast<uint32_t>(kMixB >> 32) +
         zh * static_cast<uint32_t>(kMixB);
}

__device__ __forceinline__ uint32_t phi_pre(uint64_t xpre, uint64_t kpre, uint32_t m) {
  return __umulhi(family_top32(xpre, kpre), m);
}

// The same for a range fixed at compile time: for m = 2^k,
// floor(h * 2^k / 2^32) is the top k bits of h (a shift, no multiply).
__host__ __device__ constexpr int log2_exact(int m) { return m <= 1 ? 0 : 1 + log2_exact(m >> 1); }

template <int M>
__device__ __forceinline__ uint32_t phi_fixed(uint64_t xpre, uint64_t kpre) {
  const uint32_t h = family_top32(xpre, kpre);
  if constexpr (M >= 2 && (M & (M - 1)) == 0)
    return h >> (32 - log2_exact(M));
  else
    return __umulhi(h, static_cast<uint32_t>(M));
}

// ---------------------------------------------------------------- bit arrays
// Bit k of an array is bit (k mod 64) of word k / 64.
__device__ __forceinline__ uint64_t read_bits(const uint64_t* a, uint64_t pos, uint32_t width) {
  if (width == 0) return 0;
  const uint64_t w = pos >> 6;
  const uint32_t o = static_cast<uint32_t>(pos & 63);
  uint64_t v = __ldg(a + w) >> o;
  if (o + width > 64) v |= __ldg(a + w + 1) << (64 - o);
  return width == 64 ? v : (v & ((1ull << width) - 1));
}

// Position of the set bit of rank k (0-based) in a 64-bit word (k < popc).
__device__ __forceinline__ uint32_t select_in_word(uint64_t word, uint32_t k) {
  uint32_t pos = 0;
  uint32_t lo = static_cast<uint32_t>(word);
  uint32_t c = __popc(lo);
  uint32_t w = lo;
  if (k >= c) {
    k -= c;
    pos = 32;
    w = static_cast<uint32_t>(word >> 32);
  }
  c = __popc(w & 0xFFFFu);
  if (k >= c) { k -= c; pos += 16; w >>= 16; }
  c = __popc(w & 0xFFu);
  if (k >= c) { k -= c; pos += 8; w >>= 8; }
  c = __popc(w & 0xFu);
  if (k >= c) { k -= c; pos += 4; w >>= 4; }
  c = __popc(w & 0x3u);
  if (k >= c) { k -= c; pos += 2; w >>= 2; }
  c = w & 1u;
  if (k >= c) pos += 1;
  return pos;
}

// Position of the one of rank `rank` (0-based) counting from the one at
// position `pos` (rank 0), scanning words.
__device__ __forceinline__ uint64_t select_from(const uint64_t* a, uint64_t pos, uint64_t rank) {
  uint64_t w = pos >> 6;
  uint64_t word = __ldg(a + w) & (~0ull << (pos & 63));
  for (;;) {
    const uint32_t c = __popcll(word);
    if (rank < c) break;
    rank -= c;
    word = __ldg(a + (++w));
  }
  return (w << 6) + select_in_word(word, static_cast<uint32_t>(rank));
}

// Position of the first one at or after `pos`.
__device__ __forceinline__ uint64_t next_one(const uint64_t* a, uint64_t pos) {
  uint64_t w = pos >> 6;
  uint64_t word = __ldg(a + w) & (~0ull << (pos & 63));
  while (!word) word = __ldg(a + (++w));
  return (w << 6) + static_cast<uint64_t>(__ffsll(static_cast<long long>(word)) - 1);
}

// Sec. 7.4: position of the one of rank i in upper-bits list `list` (0 for
// prefix sums, 1 for offsets), from the u64 anchor of its 2^14 block and the
// u16 offset of its 2^8 block (0xFFFF = did not fit: use an earlier one).
__device__ __forceinline__ uint64_t ef_select(const View& v, int list, uint64_t i) {
  const uint64_t* up = list ? v.upper_b : v.upper_a;
  const uint64_t k = i >> kInvHi;
  uint64_t j = i >> kInvLo;
  const uint64_t first = k << (kInvHi - kInvLo);
  uint32_t sub = v.subs[2 * j + list];
  while (sub == 0xFFFFu && j > first) {
    j--;
    sub = v.subs[2 * j + list];
  }
  const uint64_t pos = __ldg(v.anchors + 2 * k + list) + sub;
  return select_from(up, pos, i - (j << kInvLo));
}

}  // namespace rs
