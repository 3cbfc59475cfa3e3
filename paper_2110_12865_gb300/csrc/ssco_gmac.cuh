// ssco_gmac.cuh -- the gather-multiply-accumulate core shared by the
// assembly groups and the sparse-expression levels (Sec. 4.3 / 4.4: the
// members of one group share the structure of their expression and differ
// only in their harvested leaves).
//
// A group's members all have the same number of terms; its index tables
// are term-major with the member innermost (term t of member i at
// t * stride + i), so the lanes of a warp read one contiguous run per term.
// A group whose coefficients are all equal keeps one constant instead of a
// coefficient table (the sum is then scaled once).  With kSecond each term
// is the product of two gathered values, otherwise of one.
#pragma once
#include <cstdint>

namespace ssco {

template <class Acc, bool kSecond, class Load>
__device__ __forceinline__ Acc gmac(Acc acc, int nterms, int64_t stride, const int32_t* __restrict__ i1,
                                    const int32_t* __restrict__ i2, const Acc* __restrict__ coef, Acc c_uniform,
                                    Load load) {
    if (coef == nullptr) {
        Acc s = Acc(0);
        for (int t = 0; t < nterms; ++t) {
            Acc p = load(i1[(int64_t)t * stride]);
            if (kSecond) p *= load(i2[(int64_t)t * stride]);
            s += p;
        }
        acc += c_uniform * s;
    } else {
        for (int t = 0; t < nterms; ++t) {
            Acc p = load(i1[(int64_t)t * stride]);
            if (kSecond) p *= load(i2[(int64_t)t * stride]);
            acc += coef[(int64_t)t * stride] * p;
        }
    }
    return acc;
}

}  // namespace ssco
