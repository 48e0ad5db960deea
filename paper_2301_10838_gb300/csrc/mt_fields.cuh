// Where a CTA's work lives: one field (the descriptor travels by value in the
// kernel parameters) or a packed batch of fields (a descriptor table in the
// workspace, searched by the first tile / first compaction chunk of each
// field). Every kernel of the path is written once against this interface.
#pragma once
#include <cstdint>

#include "mt_internal.h"

namespace mt {

struct OneField {
    FieldDesc d;
    __device__ __forceinline__ FieldDesc tile(uint32_t g, uint32_t &local) const
    {
        local = g;
        return d;
    }
    __device__ __forceinline__ FieldDesc chunk(uint64_t g, uint64_t &local, uint32_t &fi) const
    {
        local = g;
        fi = 0;
        return d;
    }
    __device__ __forceinline__ FieldDesc field(uint32_t) const { return d; }
};

struct ManyFields {
    const FieldDesc *d;
    uint32_t nfields;
    // last field whose first tile is <= g (fields with no tiles cannot occur)
    __device__ __forceinline__ FieldDesc tile(uint32_t g, uint32_t &local) const
    {
        uint32_t lo = 0, hi = nfields;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (d[mid].tile0 <= g) lo = mid;
            else hi = mid;
        }
        local = g - d[lo].tile0;
        return d[lo];
    }
    __device__ __forceinline__ FieldDesc chunk(uint64_t g, uint64_t &local, uint32_t &fi) const
    {
        uint32_t lo = 0, hi = nfields;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (d[mid].chunk0 <= g) lo = mid;
            else hi = mid;
        }
        local = g - d[lo].chunk0;
        fi = lo;
        return d[lo];
    }
    __device__ __forceinline__ FieldDesc field(uint32_t i) const { return d[i]; }
};

}  // namespace mt
