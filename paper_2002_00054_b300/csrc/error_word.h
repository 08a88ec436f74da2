// error_word.h -- the bits of the library's device error word (flags[FLAG_ERR])
// and their mapping to the nnp_status codes of include/nnp.h.  Plain C++ with
// no CUDA, so that the mapping compiles and can be checked on a host without a
// GPU; the kernels include it through common.cuh.
#pragma once
#include <cstddef>
#include <cstdio>

#include "../../include/nnp.h"

// Each condition has a bit of its own; kernels atomicOr them into the word.
#define ERR_NEIGH_OVERFLOW 1   // a neighbour-list row exceeds max_neighbors
#define ERR_CELL_OVERFLOW 2    // a cell of the binning holds more than its capacity
#define ERR_NONFINITE 4        // non-finite position, energy or force; invalid element type
#define ERR_CLOSE 8            // two atoms closer than 1e-4 A
#define ERR_REV 16             // reverse index: a list entry without its mirror
#define ERR_RC_OVERFLOW 32     // wide-capacity pass overflowed (internal)
#define ERR_RANGE 64           // a force contribution non-finite or beyond the fixed-point range
#define ERR_TIMEOUT 128        // a bounded wait of the tensor-core network ran out
#define ERR_ALL_BITS 255

// Status of a non-zero error word; writes the message into msg[len].  When
// several bits are set, the cause that explains the others is reported: input
// capacities first, then a failed wait (whose outputs are undefined), then the
// numerical conditions.
static inline int error_word_status(int f, int max_neighbors, int cell_cap, double fx_limit, char* msg, size_t len)
{
    if (f & ERR_NEIGH_OVERFLOW) {
        snprintf(msg, len, "an atom has more than max_neighbors = %d neighbours within cutoff + skin", max_neighbors);
        return NNP_ENEIGH_OVERFLOW;
    }
    if (f & ERR_CELL_OVERFLOW) {
        snprintf(msg, len, "a cell holds more than %d atoms", cell_cap);
        return NNP_ENEIGH_OVERFLOW;
    }
    if (f & ERR_RC_OVERFLOW) {
        snprintf(msg, len, "internal error: wide-capacity pass overflowed");
        return NNP_ECUDA;
    }
    if (f & ERR_TIMEOUT) {
        snprintf(msg, len,
                 "tensor-core network: a bounded wait for an MMA to complete ran out; the call's outputs are "
                 "undefined");
        return NNP_ECUDA;
    }
    if (f & ERR_RANGE) {
        snprintf(msg, len, "a force contribution is non-finite or exceeds %g eV/A", fx_limit);
        return NNP_ENONFINITE;
    }
    if (f & ERR_CLOSE) {
        snprintf(msg, len, "two atoms are closer than 1e-4 A");
        return NNP_ENONFINITE;
    }
    if (f & ERR_NONFINITE) {
        snprintf(msg, len, "non-finite position/energy/force or invalid element type");
        return NNP_ENONFINITE;
    }
    if (f & ERR_REV) {
        snprintf(msg, len, "internal error: neighbour list not symmetric");
        return NNP_ECUDA;
    }
    snprintf(msg, len, "device error word 0x%x", f);
    return NNP_ECUDA;
}
