// smem_layout.h -- dynamic shared-memory layout of the tile kernel, used by
// the host (to size the launch and to cap the half-path entries of a tile)
// and by the device code (to carve the buffer).  Pure integer arithmetic.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define PARS3_HD __host__ __device__ __forceinline__
#else
#define PARS3_HD inline
#endif

namespace pars3 {

// Dynamic shared memory of the tile kernel.  A tile block holds the x
// window, the tile's middle entries (filled by TMA bulk copies) and scratch;
// a block of long-row pieces uses none.
struct SmemLayout {
    uint32_t xs, rowacc, colacc, hval, hcol, cperm, hrowc, hrp, hcs, red, mbar, total;
};

PARS3_HD uint32_t align128(uint32_t a) { return (a + 127u) & ~127u; }

// T: tile rows, W: window, Mh: half-path entries of the largest tile (padded
// to 8; 0 when no tile stages middle entries, and then only the row sums and
// the reduction area remain, so that the rest of the SM's shared memory
// serves as L1), CS: column segment words of the largest tile (a multiple of
// 4), vsz/xsz/asz: bytes of the value, vector and accumulator types.  Every
// region starts on a 128-byte boundary (TMA bulk copies need 16).
PARS3_HD SmemLayout smem_layout(uint32_t T, uint32_t W, uint32_t Mh, uint32_t CS, uint32_t vsz, uint32_t xsz,
                                uint32_t asz) {
    SmemLayout s;
    const uint32_t half = Mh > 0 ? 1u : 0u;
    s.xs = 0;
    s.rowacc = align128(s.xs + half * (T + W) * xsz);
    s.colacc = align128(s.rowacc + T * asz);
    s.hval = align128(s.colacc + half * T * asz);
    s.hcol = align128(s.hval + Mh * vsz);
    s.cperm = align128(s.hcol + Mh * 2u);
    s.hrowc = align128(s.cperm + Mh * 2u);
    s.hrp = align128(s.hrowc + Mh * 2u);
    s.hcs = align128(s.hrp + half * (T + 8u) * 2u);
    s.red = align128(s.hcs + half * CS * 4u);
    s.mbar = align128(s.red + 32u * 8u);
    s.total = align128(s.mbar + 8u);
    return s;
}

}  // namespace pars3
