// gfip_grouped.h -- descriptors of the grouped GEMM shared by the launcher and the C ABI.
#pragma once

#include <cstdint>

#include "gfip_internal.h"

namespace gfip {

template <typename T> struct GroupDesc {
    const T *A;
    const T *B;
    T *C;
    int64_t lda, ldb, ldc;
    int m, n, k, kt;      // kt = 0 when A and B are not to be read (alpha == 0 or k == 0)
    int mt;               // tile rows
    int order;            // bit 0: op(A) rows run along memory, bit 1: op(B) columns do
    T alpha, beta;
};

template <typename T> struct GroupParams {
    int count;
    const char *transa, *transb;
    const int *m, *n, *k;
    const T *alpha, *beta;
    const T *const *A;
    const T *const *B;
    T *const *C;
    const int64_t *lda, *ldb, *ldc;
    GroupDesc<T> *desc;   // [count]
    int *prefix;          // [count + 1]: prefix[g] = first tile of problem g, prefix[count] = total
    unsigned int *status;
};

}  // namespace gfip
