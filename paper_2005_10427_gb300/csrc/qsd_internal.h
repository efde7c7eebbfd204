// Internal structures shared by the planner, the executor and the kernels.
#pragma once

#include <stdint.h>

#include "qsd.h"

namespace qsd {

constexpr int kMaxOrder = QSD_MAX_ORDER;
constexpr int kMaxFields = 8;   // key modes one radix digit can span
constexpr int kMaxPasses = 32;  // 8 modes x 31 bits / 8-bit digits, rounded up
constexpr int kRadixBits = 8;   // widest digit of any pass
constexpr int kRadix = 1 << kRadixBits;

// One slice of a radix digit: bits [shift, shift + width) of coordinate
// `mode`, placed at bit `dst` of the digit.
struct DigitField {
  int8_t mode;
  int8_t shift;
  int8_t width;
  int8_t dst;
};

// One stable radix pass: digit = OR of the fields (at most kRadixBits bits).
struct PassDesc {
  int nfields;
  int bits;
  DigitField f[kMaxFields];
};

// One execution group: a stable sort of every bucket of equal prefix
// coordinates by the packed key of `key_modes` (most significant first),
// run as `npasses` least-significant-digit-first radix passes. It stands
// for the PartialSort calls of Algorithm 3 that share one prefix.
struct Group {
  int prefix_len;
  int prefix_modes[kMaxOrder];
  int nkeys;
  int key_modes[kMaxOrder];
  int key_bits;
  int npasses;
  PassDesc pass[kMaxPasses];
  // (key, index) form: the packed key's words and the entry index are the
  // rows the passes sort; kpass[p] is pass p with its fields naming key
  // words instead of modes. Key mode i sits at bits [kbase[i], kbase[i] +
  // kwidth[i]) of the key.
  int key_index;
  int key_words;  // 1 (key <= 32 bits) or 2
  int kbase[kMaxOrder];
  int kwidth[kMaxOrder];
  PassDesc kpass[kMaxPasses];
};

}  // namespace qsd

struct qsd_plan_s {
  int order;
  int64_t dims[QSD_MAX_ORDER];
  int tau[QSD_MAX_ORDER];
  int sigma[QSD_MAX_ORDER];
  int ncalls;
  int nbucketed;
  int call_prefix_len[QSD_MAX_ORDER];
  int call_mode[QSD_MAX_ORDER];
  int ngroups;
  qsd::Group groups[QSD_MAX_ORDER];
  qsd_plan_options opts;
  int local_capacity;  // entries per shared-memory bucket sort
  int digit_bits;      // widest digit of the global passes
};
