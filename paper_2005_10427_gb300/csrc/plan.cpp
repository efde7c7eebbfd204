// Host pass planner: Algorithm 3 (QuesadillaSort, Section 3.5) plus the
// bit-packed key and radix-digit schedule that the kernels execute.
//
// The paper-level plan is the list of PartialSort calls Algorithm 3 makes.
// Calls that share the prefix (sigma_1..sigma_l) run back to back in its
// inner sort loop, sorting sigma_k, sigma_{k-1}, ..., sigma_{l+1}; because
// each is stable, together they are one stable sort of every bucket of equal
// prefix by the key (sigma_{l+1}, ..., sigma_k), most significant first.
// That is an execution "group". Its key is packed from ceil(log2 n_m)-bit
// fields (bit-packing and sub-mode radix digits are the improvements the
// paper's conclusion proposes) and sorted least significant digit first.
#include <algorithm>
#include <cstring>
#include <new>

#include "qsd_internal.h"

namespace {

int mode_bits(int64_t dim) {
  int b = 0;
  while (b < 62 && (int64_t(1) << b) < dim) ++b;
  return b;  // 0 for dim == 1
}

bool is_perm(int order, const int* p) {
  if (!p) return false;
  bool seen[QSD_MAX_ORDER] = {false};
  for (int i = 0; i < order; ++i) {
    if (p[i] < 0 || p[i] >= order || seen[p[i]]) return false;
    seen[p[i]] = true;
  }
  return true;
}

// Splits the packed key of group g into LSD-first digit passes of at most
// `digit_bits` bits, as even as possible; with first_bits (0 < first_bits <
// digit_bits) the least significant digit takes first_bits bits and the
// rest is split evenly, when that needs no more passes than the even split
// (a narrower first digit spreads each tile over fewer runs where the key's
// low bits are near uniform). False when the passes exceed what a group
// holds.
bool schedule_digits(const int64_t* dims, qsd::Group& g, int digit_bits, int first_bits) {
  int base[QSD_MAX_ORDER], width[QSD_MAX_ORDER];
  int acc = 0;
  for (int i = g.nkeys - 1; i >= 0; --i) {  // last key mode = lowest bits
    width[i] = mode_bits(dims[g.key_modes[i]]);
    base[i] = acc;
    acc += width[i];
  }
  g.key_bits = acc;
  if (acc == 0) {
    g.npasses = 0;
    return true;
  }
  int np = (acc + digit_bits - 1) / digit_bits;
  if (np > qsd::kMaxPasses) return false;
  // the first digit's width, then the rest split evenly over np - 1 passes
  int first = 0;
  if (first_bits > 0 && first_bits < digit_bits && np >= 2 &&
      1 + (acc - first_bits + digit_bits - 1) / digit_bits <= np)
    first = first_bits;
  g.npasses = np;
  int lo = 0;
  for (int p = 0; p < np; ++p) {
    int bits;
    if (first) {
      const int rest = acc - first, nr = np - 1;
      bits = p == 0 ? first : rest / nr + (p - 1 < rest % nr ? 1 : 0);
    } else {
      bits = acc / np + (p < acc % np ? 1 : 0);
    }
    int hi = lo + bits;
    qsd::PassDesc& d = g.pass[p];
    d.nfields = 0;
    d.bits = bits;
    for (int i = g.nkeys - 1; i >= 0; --i) {
      int a = std::max(lo, base[i]);
      int b = std::min(hi, base[i] + width[i]);
      if (a >= b) continue;
      qsd::DigitField& f = d.f[d.nfields++];
      f.mode = (int8_t)g.key_modes[i];
      f.shift = (int8_t)(a - base[i]);
      f.width = (int8_t)(b - a);
      f.dst = (int8_t)(a - lo);
    }
    lo = hi;
  }
  return true;
}

// (key, index) form of a group without a prefix whose packed key fits 64
// bits and takes two or more passes: the same digit passes, re-expressed on
// the rows the pack kernel writes (key bits 0..31 in word 0, bits 32..63 in
// word 1, then the entry index). The plain passes stay for the paths that
// sort whole entries (a tensor small enough for one block, batches).
void to_key_index(const int64_t* dims, qsd::Group& g) {
  if (g.prefix_len != 0 || g.npasses < 2 || g.key_bits > 64) return;
  int acc = 0;
  for (int i = g.nkeys - 1; i >= 0; --i) {  // last key mode = lowest bits
    g.kwidth[i] = mode_bits(dims[g.key_modes[i]]);
    g.kbase[i] = acc;
    acc += g.kwidth[i];
  }
  g.key_index = 1;
  g.key_words = g.key_bits > 32 ? 2 : 1;
  int lo = 0;
  for (int p = 0; p < g.npasses; ++p) {
    qsd::PassDesc& d = g.kpass[p];
    d.bits = g.pass[p].bits;
    const int hi = lo + d.bits;
    d.nfields = 0;
    for (int w = 0; w < 2; ++w) {
      const int a = std::max(lo, 32 * w), b = std::min(hi, 32 * w + 32);
      if (a >= b) continue;
      qsd::DigitField& f = d.f[d.nfields++];
      f.mode = (int8_t)w;
      f.shift = (int8_t)(a - 32 * w);
      f.width = (int8_t)(b - a);
      f.dst = (int8_t)(a - lo);
    }
    lo = hi;
  }
}

}  // namespace

extern "C" {

qsd_status qsd_plan_ex(int order, const int64_t* dims,
                       const int* input_mode_order, const int* target_perm,
                       const qsd_plan_options* opts, qsd_plan_t* out) {
  if (!out) return QSD_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (order < 1) return QSD_ERR_INVALID_ARGUMENT;
  if (order > QSD_MAX_ORDER) return QSD_ERR_UNSUPPORTED;
  if (!dims) return QSD_ERR_INVALID_ARGUMENT;
  for (int m = 0; m < order; ++m)
    if (dims[m] < 1 || dims[m] > 2147483647LL) return QSD_ERR_INVALID_ARGUMENT;
  if (!is_perm(order, input_mode_order) || !is_perm(order, target_perm))
    return QSD_ERR_INVALID_ARGUMENT;
  qsd_plan_options o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.digit_bits < 0 || o.digit_bits > qsd::kRadixBits)
    return QSD_ERR_INVALID_ARGUMENT;
  if (o.local_capacity != 0 && o.local_capacity != 1024 &&
      o.local_capacity != 2048 && o.local_capacity != 4096 &&
      o.local_capacity != 8192)
    return QSD_ERR_INVALID_ARGUMENT;
  if (o.tile != 0 && o.tile != 1024 && o.tile != 2048 && o.tile != 3584 && o.tile != 4096)
    return QSD_ERR_INVALID_ARGUMENT;
  if (o.chunk_tiles < 0 || o.chunk_tiles > 256) return QSD_ERR_INVALID_ARGUMENT;
  if (o.top_k < 0 || o.top_k > QSD_MAX_ORDER) return QSD_ERR_INVALID_ARGUMENT;
  if (o.first_digit_bits < 0 || o.first_digit_bits > qsd::kRadixBits)
    return QSD_ERR_INVALID_ARGUMENT;

  qsd_plan_s* p = new (std::nothrow) qsd_plan_s;
  if (!p) return QSD_ERR_OUT_OF_MEMORY;
  std::memset(p, 0, sizeof(*p));
  p->order = order;
  p->opts = o;
  for (int m = 0; m < order; ++m) {
    p->dims[m] = dims[m];
    p->tau[m] = input_mode_order[m];
    p->sigma[m] = target_perm[m];
  }
  p->digit_bits = o.digit_bits ? o.digit_bits : qsd::kRadixBits;
  p->local_capacity = o.local_capacity ? o.local_capacity : 4096;

  // Top-K-sadilla (Section 3.6): Algorithm 3 sorts only to the order of the
  // first K target modes -- the ordering sigma_1..sigma_K followed by the
  // other modes in their tau order, where a stable sort by the K modes leaves
  // them (none of them then needs a call) -- and one last group sorts every
  // bucket of equal (sigma_1..sigma_K) completely by the remaining target
  // modes. K >= order - 1 is Quesadilla itself.
  const int K = (o.top_k > 0 && o.top_k < order - 1) ? o.top_k : order;
  int tgt[QSD_MAX_ORDER];  // the ordering Algorithm 3 sorts to
  {
    unsigned head = 0;
    for (int i = 0; i < order; ++i) {
      tgt[i] = target_perm[i];
      if (i < K) head |= 1u << target_perm[i];
    }
    int n = K < order ? K : order;
    for (int i = 0; i < order && K < order; ++i)
      if (!(head >> input_mode_order[i] & 1u)) tgt[n++] = input_mode_order[i];
  }
  bool topk_group = false;
  for (int i = 0; i < order; ++i) topk_group |= tgt[i] != target_perm[i];

  // f(tau, m) and f(sigma, m) as bit sets: the modes after m (Section 3.4).
  unsigned f_tau[QSD_MAX_ORDER] = {0}, f_sigma[QSD_MAX_ORDER] = {0};
  for (int i = 0; i < order; ++i)
    for (int j = i + 1; j < order; ++j) {
      f_tau[input_mode_order[i]] |= 1u << input_mode_order[j];
      f_sigma[tgt[i]] |= 1u << tgt[j];
    }
  auto needs_sort = [&](int m) {  // f(sigma, m) not a subset of f(tau, m)
    return (f_sigma[m] & ~f_tau[m]) != 0;
  };
  auto s = [&](int i) { return tgt[i - 1]; };  // sigma_i, 1-based

  if (o.no_skip) {
    // Full LSD radix sort over every mode: r non-bucketed calls, sigma_r
    // first (Section 3's baseline that skipping improves on).
    for (int k = order; k >= 1; --k) {
      p->call_prefix_len[p->ncalls] = 0;
      p->call_mode[p->ncalls++] = s(k);
    }
    qsd::Group& g = p->groups[p->ngroups++];
    g.prefix_len = 0;
    g.nkeys = order;
    for (int i = 0; i < order; ++i) g.key_modes[i] = target_perm[i];
  } else {
    // Algorithm 3 with 1-based l, k as printed.
    int l = 0;
    while (l < order) {
      int k = l;
      while (k + 1 < order && needs_sort(s(k + 1))) ++k;
      int l_next = k + 1;
      if (k > l) {
        qsd::Group& g = p->groups[p->ngroups++];
        g.prefix_len = l;
        for (int i = 0; i < l; ++i) g.prefix_modes[i] = s(i + 1);
        g.nkeys = k - l;
        for (int i = 0; i < k - l; ++i) g.key_modes[i] = s(l + 1 + i);
      }
      for (int kk = k; kk > l; --kk) {  // the sort loop: sigma_k down to sigma_{l+1}
        p->call_prefix_len[p->ncalls] = l;
        p->call_mode[p->ncalls++] = s(kk);
        if (l > 0) p->nbucketed++;
      }
      l = l_next;
    }
    if (topk_group) {  // Top-K-sadilla's complete sort of every bucket
      qsd::Group& g = p->groups[p->ngroups++];
      g.prefix_len = K;
      for (int i = 0; i < K; ++i) g.prefix_modes[i] = target_perm[i];
      g.nkeys = order - K;
      for (int i = K; i < order; ++i) g.key_modes[i - K] = target_perm[i];
    }
    if (o.global_groups) {
      // An equivalent execution: the input of a group is already sorted by
      // its prefix, so one stable sort of the whole tensor by (prefix, key)
      // gives what sorting every bucket by the key gives -- with more digit
      // passes but no bucket discovery or bucket sort.
      for (int gi = 0; gi < p->ngroups; ++gi) {
        qsd::Group& g = p->groups[gi];
        if (g.prefix_len == 0) continue;
        int keys[QSD_MAX_ORDER];
        int nk = 0;
        for (int i = 0; i < g.prefix_len; ++i) keys[nk++] = g.prefix_modes[i];
        for (int i = 0; i < g.nkeys; ++i) keys[nk++] = g.key_modes[i];
        g.nkeys = nk;
        for (int i = 0; i < nk; ++i) g.key_modes[i] = keys[i];
        g.prefix_len = 0;
      }
    }
  }
  for (int i = 0; i < p->ngroups; ++i)
    if (!schedule_digits(p->dims, p->groups[i], p->digit_bits, o.first_digit_bits)) {
      delete p;
      return QSD_ERR_UNSUPPORTED;  // a key too wide for the digit width
    }
  if (o.key_index)
    for (int i = 0; i < p->ngroups; ++i) to_key_index(p->dims, p->groups[i]);
  *out = p;
  return QSD_OK;
}

qsd_status qsd_plan(int order, const int64_t* dims, const int* input_mode_order,
                    const int* target_perm, qsd_plan_t* out) {
  return qsd_plan_ex(order, dims, input_mode_order, target_perm, nullptr, out);
}

qsd_status qsd_plan_get_info(qsd_plan_t plan, qsd_plan_info* info) {
  if (!plan || !info) return QSD_ERR_INVALID_ARGUMENT;
  std::memset(info, 0, sizeof(*info));
  info->order = plan->order;
  for (int m = 0; m < plan->order; ++m) {
    info->input_mode_order[m] = plan->tau[m];
    info->target_perm[m] = plan->sigma[m];
  }
  info->num_calls = plan->ncalls;
  info->num_bucketed_calls = plan->nbucketed;
  for (int i = 0; i < plan->ncalls; ++i) {
    info->call_prefix_len[i] = plan->call_prefix_len[i];
    info->call_mode[i] = plan->call_mode[i];
  }
  info->num_groups = plan->ngroups;
  for (int g = 0; g < plan->ngroups; ++g) {
    info->group_prefix_len[g] = plan->groups[g].prefix_len;
    info->group_num_keys[g] = plan->groups[g].nkeys;
    info->group_key_bits[g] = plan->groups[g].key_bits;
    info->group_digit_passes[g] = plan->groups[g].npasses;
    info->group_key_index[g] = plan->groups[g].key_index;
  }
  info->local_capacity = plan->local_capacity;
  return QSD_OK;
}

void qsd_plan_destroy(qsd_plan_t plan) { delete plan; }

const char* qsd_status_string(qsd_status status) {
  switch (status) {
    case QSD_OK: return "QSD_OK";
    case QSD_ERR_INVALID_ARGUMENT: return "QSD_ERR_INVALID_ARGUMENT";
    case QSD_ERR_UNSUPPORTED: return "QSD_ERR_UNSUPPORTED";
    case QSD_ERR_OUT_OF_MEMORY: return "QSD_ERR_OUT_OF_MEMORY";
    case QSD_ERR_CUDA: return "QSD_ERR_CUDA";
    case QSD_ERR_UNSORTED_INPUT: return "QSD_ERR_UNSORTED_INPUT";
    case QSD_ERR_COORD_OUT_OF_RANGE: return "QSD_ERR_COORD_OUT_OF_RANGE";
    case QSD_ERR_TIMEOUT: return "QSD_ERR_TIMEOUT";
    case QSD_ERR_BUDGET: return "QSD_ERR_BUDGET";
    case QSD_ERR_WORKSPACE_TOO_SMALL: return "QSD_ERR_WORKSPACE_TOO_SMALL";
  }
  return "QSD_ERR_UNKNOWN";
}

const char* qsd_version(void) { return "qsd 0.1.0 (sm_103a)"; }

}  // extern "C"
