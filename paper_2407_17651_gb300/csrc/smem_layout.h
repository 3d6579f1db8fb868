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

// Dynamic shared memory of the persistent tile kernel: kStages staging
// buffers (everything a tile or a long-row chunk reads contiguously, filled
// by TMA bulk copies) followed by per-block scratch.
struct StageLayout {  // offsets inside one stage
    uint32_t xs, hrp, hval, hcol, cperm, fmeta, fval, fcol, bytes;
};
struct SmemLayout {
    StageLayout st;
    uint32_t stage_bytes;          // stride between stages
    uint32_t rowacc, q, cs, ce, mbar, total;
};

PARS3_HD uint32_t align128(uint32_t a) { return (a + 127u) & ~127u; }

// T: tile rows, W: window, Mh: half-path entries of the largest tile (padded
// to 8), S: sliced-ELL slices of the largest tile, F: sliced-ELL entries of
// the largest tile or of a long-row chunk with alignment slack, vsz/xsz/asz:
// bytes of the value, vector and accumulator types.  Every region starts on
// a 128-byte boundary (TMA bulk copies need 16).
PARS3_HD SmemLayout smem_layout(uint32_t T, uint32_t W, uint32_t Mh, uint32_t S, uint32_t F, uint32_t vsz,
                                uint32_t xsz, uint32_t asz) {
    SmemLayout s;
    StageLayout &g = s.st;
    g.xs = 0;
    g.hrp = align128(g.xs + (T + W) * xsz);
    g.hval = align128(g.hrp + (T + 8u) * 2u);
    g.hcol = align128(g.hval + Mh * vsz);
    g.cperm = align128(g.hcol + Mh * 2u);
    g.fmeta = align128(g.cperm + Mh * 2u);
    g.fval = align128(g.fmeta + S * 32u * 4u);
    g.fcol = align128(g.fval + F * vsz);
    g.bytes = align128(g.fcol + F * 4u);
    s.stage_bytes = g.bytes;
    const uint32_t base = 2u * s.stage_bytes;
    s.rowacc = base;
    s.q = align128(s.rowacc + T * asz);
    s.cs = align128(s.q + (vsz == asz ? 0u : Mh * asz));
    s.ce = align128(s.cs + (T + W) * 2u);
    s.mbar = align128(s.ce + (T + W) * 2u);
    s.total = align128(s.mbar + 2u * 8u);
    return s;
}

}  // namespace pars3
