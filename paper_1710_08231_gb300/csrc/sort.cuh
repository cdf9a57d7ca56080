// sort.cuh -- device-wide radix sort.
#pragma once

#include "gp_internal.cuh"

namespace gp {

// Stable LSD radix sort of n (key, value) pairs by the low `bits` key bits. The sorted pairs end in
// (keys_tmp, vals_tmp) when *result_in_tmp is true on return, else in (keys, vals).
int radix_sort_pairs(unsigned long long *keys, unsigned long long *vals, unsigned long long *keys_tmp,
                     unsigned long long *vals_tmp, int64_t n, int bits, bool *result_in_tmp, Workspace &ws);

}  // namespace gp
