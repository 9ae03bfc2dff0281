// sv_check.cuh -- the checked build.  Compiled with -DSV_CHECK=1 (build(check=True),
// libsv_gb300_check.so), the kernels that index through host-built tables -- sector
// pair lists, string ranks, gather tables, product-plane offsets -- test each index
// they compute against the size of the buffer it addresses before the access.  A bad
// index skips the access (a load yields zero) and sets a bit in this translation
// unit's check word instead of faulting; sv_check_status() returns the words of every
// unit and clears them.  The default build compiles every check to `true`.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#ifndef SV_CHECK
#define SV_CHECK 0
#endif

// Bits of the check word: which kind of index was out of range.
enum : uint32_t {
    kChkPair = 1u << 0,    // sector pair address (pair lists)
    kChkRank = 1u << 1,    // string rank / partner row
    kChkGather = 1u << 2,  // shared-memory gather offset (tables)
    kChkPlane = 1u << 3,   // product-plane or compact-matrix offset
};

#if SV_CHECK
namespace {
__device__ unsigned int sv_check_word;  // one per translation unit
}
// true when i < n; else records `bit` and returns false (the caller skips the access)
#define SV_IN_RANGE(i, n, bit) \
    (((size_t)(i) < (size_t)(n)) ? true : (atomicOr(&sv_check_word, (unsigned int)(bit)), false))
// This unit's word (read and cleared), for sv_check_status.
#define SV_CHECK_READER(name)                                                                         \
    uint32_t name() {                                                                                 \
        unsigned int w = 0, z = 0;                                                                    \
        if (cudaMemcpyFromSymbol(&w, sv_check_word, sizeof(w)) != cudaSuccess) return 0x80000000u;   \
        if (cudaMemcpyToSymbol(sv_check_word, &z, sizeof(z)) != cudaSuccess) return 0x80000000u;      \
        return w;                                                                                     \
    }
#else
#define SV_IN_RANGE(i, n, bit) true
#define SV_CHECK_READER(name) \
    uint32_t name() { return 0; }
#endif
