// gfip_grouped.h -- descriptors of the grouped GEMM shared by the launcher and the C ABI.
#pragma once

#include <cstdint>

#include "gfip_internal.h"

namespace gfip {

// One problem of a grouped launch, as the prepare kernel leaves it for the GEMM kernel.
template <typename T> struct GroupDesc {
    const T *A;
    const T *B;
    T *C;
    int64_t lda, ldb, ldc;
    int m, n, k;
    int mt, nt;        // warp tiles along m and n (of the problem's tile shape)
    int shape;         // tile shape (GFIP_GROUP_TILE_*)
    int splits;        // k-split factor: each tile is computed in `splits` k-ranges
    int ks;            // k rows per split (a multiple of the k chunk), or 0 (A, B not read)
    int order;         // bit 0: op(A) rows run along memory ('N'), bit 1: op(B) cols do ('T')
    int ctr_off;       // first arrival counter of this problem's split tiles
    int64_t part_off;  // first partial-sum element of this problem's split tiles
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
    const int *plan;      // [count] shape | splits << 8 per problem, or null (uniform)
    const int *order;     // [count] processing order (problem index per rank), or null
    int uniform_shape;    // the shape of every problem when plan is null
    GroupDesc<T> *desc;   // [count], by rank (processing order)
    int *units;           // [count] work units (tiles x splits) per rank
    int *stiles;          // [count] split tiles per rank
    int64_t *pelems;      // [count] partial-sum elements per rank
    int *prefix;          // [count + 1] first unit of each rank, total at [count]
    int *counters;        // [max_split_tiles] arrival counters of split tiles
    int max_split_tiles;
    T *partial;           // [partial_capacity] partial sums of split tiles
    int64_t partial_capacity;
    unsigned int *status;
};

}  // namespace gfip
