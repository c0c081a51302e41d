// Three-plane BF16 representation of FP32 values: v = hi + mid + lo, each
// plane rounded to nearest from the remainder of the previous ones (about 24
// significant bits in total).  The operand format of the split-BF16 block
// products; the product of two split values is taken as the six plane
// products with plane indices summing to at most 2.
#pragma once
#include <cuda_bf16.h>

namespace gpk {

__device__ __forceinline__ void split3(float v, __nv_bfloat16& hi, __nv_bfloat16& mid, __nv_bfloat16& lo)
{
    hi = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(hi);
    mid = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(mid);
    lo = __float2bfloat16_rn(r2);
}

}  // namespace gpk
