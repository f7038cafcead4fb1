// Host-side TMA descriptor encoding (see tensor_map.cpp).
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "radon.h"

namespace radon {

// Encodes a tiled tensor map (no swizzle, out-of-range elements read as zero).  `strides_bytes`
// holds rank-1 entries (dimension 1..rank-1).  Returns the CUresult (0 on success, -1 if the
// driver entry point is unavailable).
int encode_tiled(CUtensorMap* map, CUtensorMapDataType dt, int rank, void* base, const uint64_t* dims,
                  const uint64_t* strides_bytes, const uint32_t* box, CUtensorMapL2promotion l2);

CUtensorMapDataType tma_dtype(radon_dtype dt);

}  // namespace radon
