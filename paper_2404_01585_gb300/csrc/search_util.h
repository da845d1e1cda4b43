// Membership test in a sorted run of distinct vertex ids, shared by the search kernels and the
// host-side unit test (plain C++ when not compiled by nvcc).
//
// Interpolation search with a bisection guard: every step probes the interpolated position and
// the midpoint of the current interval together (two independent loads, one memory latency) and
// keeps the tighter interval.  On ids spread evenly over their range -- a label slice of a graph
// whose vertex numbering is unrelated to its structure -- the interpolated probe lands within a
// few places of the key, so a slice of length L is decided in about log2(log2(L)) steps; the
// midpoint probe bounds the worst case by log2(L) steps, as for plain bisection (Perl, Itai and
// Avni 1978, interpolation search; the guard is the classic combination with binary search).
#pragma once
#include <cstdint>

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#endif

namespace fx {

// True when `c` occurs among at(lo) .. at(hi - 1) (strictly increasing).  `probes` counts the
// loads made.  `at(i)` returns the id at index i.
template <class At>
__host__ __device__ inline bool interp_contains(const At &at, uint32_t lo, uint32_t hi, int32_t c,
                                                uint32_t &probes) {
    if (lo >= hi) return false;
    // closed interval [a, b] with known end values va < vb once both ends differ from c
    uint32_t a = lo, b = hi - 1;
    int32_t va = at(a), vb = at(b);
    probes += (a == b) ? 1u : 2u;
    if (c <= va) return c == va;
    if (c >= vb) return c == vb;
    // va < c < vb: an occurrence lies strictly inside (a, b)
    while (b - a > 1) {
        const uint32_t span = b - a;
        // interpolated position, strictly inside (a, b)
        const uint64_t num = (uint64_t)((int64_t)c - (int64_t)va) * (uint64_t)span;
        const uint64_t den = (uint64_t)((int64_t)vb - (int64_t)va);
        uint32_t m1 = a + (uint32_t)(num / den);
        if (m1 <= a) m1 = a + 1;
        if (m1 >= b) m1 = b - 1;
        const uint32_t m2 = a + span / 2;  // also strictly inside (a, b) since span >= 2
        const uint32_t p = m1 < m2 ? m1 : m2, q = m1 < m2 ? m2 : m1;
        const int32_t vp = at(p);
        const int32_t vq = (q != p) ? at(q) : vp;
        probes += (q != p) ? 2u : 1u;
        if (vp == c || vq == c) return true;
        if (c < vp) {
            b = p;
            vb = vp;
        } else if (c < vq) {
            a = p;
            va = vp;
            b = q;
            vb = vq;
        } else {
            a = q;
            va = vq;
        }
    }
    return false;
}

}  // namespace fx
