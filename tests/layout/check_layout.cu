// Host-only checks of the kernel-pool and node-vector layouts the FP32 sweeps rely on
// (compiled with nvcc, run without a GPU).  Prints "OK" or the first failure.
#include <cstdio>
#include <vector>

#include "../../paper_2012_03667_gb300/csrc/qdse_internal.h"

using qdse::kpos;
using qdse::kRows;
using qdse::kswz;
using qdse::vpos;

static int fail(const char* what, int n, int a, int b) {
    std::printf("FAIL %s n=%d %d %d\n", what, n, a, b);
    return 1;
}

int main() {
    const int sizes[] = {1, 2, 3, 4, 5, 6, 7, 8, 37, 40, 64, 127, 128, 130, 384, 509, 512};
    for (int n : sizes) {
        const int ld = (n + 3) & ~3;
        const long long total = 3LL * n * ld;
        // a bijection of (row, plane, column) onto [k_off, k_off + 3 n ld)
        std::vector<int> hit(total, 0);
        for (int i = 0; i < n; ++i)
            for (int p = 0; p < 3; ++p)
                for (int j = 0; j < ld; ++j) {
                    const long long o = kpos(100, n, ld, i, p, j) - 100;
                    if (o < 0 || o >= total) return fail("range", n, i, j);
                    if (hit[o]++) return fail("collision", n, i, j);
                }
        // every 4-aligned column range of a group is one contiguous run starting at
        // kbase + (c0 / 4) * 3 nr * 4, and the 4 columns of a block are adjacent
        for (int i0 = 0; i0 < n; i0 += kRows) {
            const int nr = n - i0 < kRows ? n - i0 : kRows;
            const long long kbase = 3LL * i0 * ld;
            for (int c0 = 0; c0 < ld; c0 += 4) {
                for (int c1 = c0 + 4; c1 <= ld && c1 <= c0 + 132; c1 += 4) {
                    const long long start = kbase + (long long)(c0 >> 2) * 3 * nr * 4;
                    const long long len = (long long)(c1 - c0) * 3 * nr;
                    std::vector<int> seen(len, 0);
                    for (int r = 0; r < nr; ++r)
                        for (int p = 0; p < 3; ++p)
                            for (int j = c0; j < c1; ++j) {
                                const long long o = kpos(0, n, ld, i0 + r, p, j) - start;
                                if (o < 0 || o >= len || seen[o]++) return fail("run", n, i0, c0);
                            }
                }
                // inside block q = c0 / 4, plane-row m = 3 r + p sits at float4 m ^ kswz(nr, q)
                for (int r = 0; r < nr; ++r)
                    for (int p = 0; p < 3; ++p) {
                        const int m = 3 * r + p, q = c0 >> 2;
                        const long long o = kpos(0, n, ld, i0 + r, p, c0);
                        const long long want = kbase + (long long)q * 3 * nr * 4 + (m ^ kswz(nr, q)) * 4;
                        if (o != want) return fail("block", n, i0 + r, c0);
                        for (int e = 1; e < 4; ++e)
                            if (kpos(0, n, ld, i0 + r, p, c0 + e) != o + e) return fail("adjacent", n, r, e);
                    }
            }
        }
    }
    // the swizzle of full groups: 16-byte reads of one plane-row from 8 consecutive blocks (one
    // per lane of a quarter warp, blocks 12 float4 apart) hit 8 different bank quads
    for (int q0 = 0; q0 < 64; ++q0)
        for (int m = 0; m < 3 * kRows; ++m) {
            int used = 0;
            for (int l = 0; l < 8; ++l) {
                const int quad = (3 * kRows * l + (m ^ kswz(kRows, q0 + l))) % 8;
                if (used & (1 << quad)) return fail("banks", kRows, q0, m);
                used |= 1 << quad;
            }
        }
    // node vectors: (node, component) onto [0, 5 nv) one-to-one; a node range starting at a
    // multiple of 4 is one run of 5 * length floats; the 5 components of a lane's 4-node block
    // are 5 float4, 20 floats apart from the next lane's
    const int nv = 1024;
    std::vector<int> vh(5 * nv, 0);
    for (int x = 0; x < nv; ++x)
        for (int c = 0; c < 5; ++c) {
            const long long o = vpos(x, c);
            if (o < 0 || o >= 5 * nv || vh[o]++) return fail("vpos", nv, x, c);
            if (vpos(x, c) != 20LL * (x / 4) + 4 * c + x % 4) return fail("vpos-form", nv, x, c);
        }
    for (int x0 = 0; x0 < nv; x0 += 4)
        for (int x1 = x0 + 4; x1 <= nv && x1 <= x0 + 64; x1 += 4) {
            long long lo = 1LL << 40, hi = -1;
            for (int x = x0; x < x1; ++x)
                for (int c = 0; c < 5; ++c) {
                    lo = vpos(x, c) < lo ? vpos(x, c) : lo;
                    hi = vpos(x, c) > hi ? vpos(x, c) : hi;
                }
            if (lo != vpos(x0, 0) || hi - lo + 1 != 5LL * (x1 - x0)) return fail("vrun", nv, x0, x1);
        }
    std::printf("OK\n");
    return 0;
}
