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

struct SmemLayout {
    uint32_t xs, rowacc, q, hcol, cperm, hrp, frp, cs, ce, carry_row, carry_val, mbar, total;
};

PARS3_HD uint32_t align16(uint32_t a) { return (a + 15u) & ~15u; }

// T: tile rows, W: window, M: half-path entries of the largest tile,
// P: threads per block, xsz/asz: bytes of the vector and accumulator types,
// k: right-hand sides held per window position.
PARS3_HD SmemLayout smem_layout(uint32_t T, uint32_t W, uint32_t M, uint32_t P, uint32_t xsz,
                                uint32_t asz, uint32_t k) {
    SmemLayout s;
    s.xs = 0;
    s.rowacc = align16(s.xs + (T + W) * xsz * k);
    s.q = align16(s.rowacc + T * asz * k);
    s.hcol = align16(s.q + M * asz * k);
    s.cperm = align16(s.hcol + M * 2u);
    s.hrp = align16(s.cperm + M * 2u);
    s.frp = align16(s.hrp + (T + 8u) * 2u);
    s.cs = align16(s.frp + (T + 8u) * 4u);
    s.ce = align16(s.cs + (T + W) * 2u);
    s.carry_row = align16(s.ce + (T + W) * 2u);
    s.carry_val = align16(s.carry_row + P * 4u);
    s.mbar = align16(s.carry_val + P * asz * k);
    s.total = align16(s.mbar + 8u);
    return s;
}

}  // namespace pars3
