// pt_host.h -- host-side helpers shared by the C-ABI runtimes (library-private):
// FP64 acceptance tables, the kernels' coupler layout, neighbour cells, and the
// host Philox used for the engineering draws.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <string>
#include <vector>

#include "pt_internal.h"

namespace ptg {

// ------------------------------------------------------------------------
// Host Philox4x32-10 for the engineering draws (Salmon et al., SC'11).
// ------------------------------------------------------------------------
inline void philox_host(const uint32_t in[4], uint32_t k0, uint32_t k1, uint32_t out[4])
{
    uint32_t c0 = in[0], c1 = in[1], c2 = in[2], c3 = in[3];
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

inline uint32_t to_u32_threshold(double p)
{
    const double x = std::floor(std::ldexp(p, 32));
    if (x >= 4294967295.0) return 0xFFFFFFFFu;
    if (x <= 0.0) return 0u;
    return (uint32_t)x;
}

inline int n_edges_of(int L) { return 16 * L * L + 8 * L * (L - 1); }

// Coupler index helpers for the documented edge order.
inline int intra_edge(int L, int cell, int kv, int kh) { (void)L; return 16 * cell + 4 * kv + kh; }
inline int vert_edge(int L, int r, int c, int k) { return 16 * L * L + (r * L + c) * 4 + k; }
inline int horiz_edge(int L, int r, int c, int k) { return 16 * L * L + 4 * L * (L - 1) + (r * (L - 1) + c) * 4 + k; }

inline uint32_t pack4(int b0, int b1, int b2, int b3)
{
    return (uint32_t)(uint8_t)(int8_t)b0 | ((uint32_t)(uint8_t)(int8_t)b1 << 8) |
           ((uint32_t)(uint8_t)(int8_t)b2 << 16) | ((uint32_t)(uint8_t)(int8_t)b3 << 24);
}

// Kernel layout of the couplers (see InstDesc): per (cell, colour), 4 words of
// negated intra-cell couplers and 4 words of negated inter-cell couplers.
inline void pack_couplers(int L, const int8_t* J, uint32_t* jw)
{
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < L; ++c) {
            const int cell = r * L + c;
            for (int col = 0; col < 2; ++col) {
                const int u = (r + c + col) & 1;
                uint32_t* w = jw + (cell * 2 + col) * 8;
                for (int k = 0; k < 4; ++k) {
                    int b[4];
                    for (int kp = 0; kp < 4; ++kp)
                        b[kp] = -(u == 0 ? J[intra_edge(L, cell, k, kp)] : J[intra_edge(L, cell, kp, k)]);
                    w[k] = pack4(b[0], b[1], b[2], b[3]);
                }
                int jm[4], jp[4];
                for (int k = 0; k < 4; ++k) {
                    if (u == 0) {
                        jm[k] = r >= 1 ? -J[vert_edge(L, r - 1, c, k)] : 0;
                        jp[k] = r + 1 < L ? -J[vert_edge(L, r, c, k)] : 0;
                    } else {
                        jm[k] = c >= 1 ? -J[horiz_edge(L, r, c - 1, k)] : 0;
                        jp[k] = c + 1 < L ? -J[horiz_edge(L, r, c, k)] : 0;
                    }
                }
                w[4] = pack4(jm[0], jp[0], 0, 0);
                w[5] = pack4(0, 0, jm[1], jp[1]);
                w[6] = pack4(jm[2], jp[2], 0, 0);
                w[7] = pack4(0, 0, jm[3], jp[3]);
            }
        }
}

inline void build_neighbours(int L, int16_t* nbr)
{
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < L; ++c) {
            const int cell = r * L + c;
            for (int col = 0; col < 2; ++col) {
                const int u = (r + c + col) & 1;
                int m = cell, p = cell;
                if (u == 0) {
                    if (r >= 1) m = (r - 1) * L + c;
                    if (r + 1 < L) p = (r + 1) * L + c;
                } else {
                    if (c >= 1) m = r * L + c - 1;
                    if (c + 1 < L) p = r * L + c + 1;
                }
                nbr[(cell * 2 + col) * 2 + 0] = (int16_t)m;
                nbr[(cell * 2 + col) * 2 + 1] = (int16_t)p;
            }
        }
}

// Largest local-field magnitude an instance can produce: max over spins of
// sum_j |J_ij| (the Metropolis table needs rows k = 0 .. K).
inline int coupler_kmax(int L, const int8_t* J)
{
    const int N = 8 * L * L;
    std::vector<int> s((size_t)N, 0);
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < L; ++c) {
            const int cell = r * L + c;
            for (int kv = 0; kv < 4; ++kv)
                for (int kh = 0; kh < 4; ++kh) {
                    const int a = std::abs((int)J[intra_edge(L, cell, kv, kh)]);
                    s[(size_t)8 * cell + kv] += a;
                    s[(size_t)8 * cell + 4 + kh] += a;
                }
            for (int k = 0; k < 4; ++k) {
                if (r + 1 < L) {
                    const int a = std::abs((int)J[vert_edge(L, r, c, k)]);
                    s[(size_t)8 * cell + k] += a;
                    s[(size_t)8 * (cell + L) + k] += a;
                }
                if (c + 1 < L) {
                    const int a = std::abs((int)J[horiz_edge(L, r, c, k)]);
                    s[(size_t)8 * cell + 4 + k] += a;
                    s[(size_t)8 * (cell + 1) + 4 + k] += a;
                }
            }
        }
    int m = 0;
    for (int v : s) m = v > m ? v : m;
    return m;
}

// Table rows for an instance: the default 19, or K + 1 rounded up to a
// multiple of 4 when its couplers need more.
inline int table_rows_for(int kmax)
{
    if (kmax + 1 <= KT_DEFAULT) return KT_DEFAULT;
    return (kmax + 1 + 3) & ~3;
}

struct Tables {
    int kt = KT_DEFAULT;           // rows per slot
    std::vector<uint32_t> thr;     // [NT][kt]
    std::vector<int64_t> xoff;     // [NT]
    std::vector<uint32_t> xthr;
    std::vector<float> xhint;      // [NT-1]
};

// Writes the FP64 acceptance tables into caller buffers, allocating nothing:
// thr [NT][kt], xoff [NT], xhint [max(NT-1, 1)], and the ragged exchange
// thresholds into xthr (capacity xcap entries; xthr NULL only counts them).
// Returns the exchange-table length, or -1 with *why set when the ladder's
// tables are too long or not monotone.
inline int64_t fill_tables(int NT, int kt, const double* betas, uint32_t* thr, int64_t* xoff, float* xhint,
                           uint32_t* xthr, int64_t xcap, const char** why)
{
    for (int t = 0; t < NT; ++t) {
        thr[(size_t)t * kt] = 0xFFFFFFFFu;   // k <= 0 always accepts; entry unused for decisions
        for (int k = 1; k < kt; ++k)
            thr[(size_t)t * kt + k] = to_u32_threshold(std::exp(-2.0 * (double)k * betas[t]));
    }
    int64_t n = 0;
    xhint[0] = 0.f;
    for (int p = 0; p + 1 < NT; ++p) {
        const double db = betas[p] - betas[p + 1];
        xoff[p] = n;
        xhint[p] = (float)(std::log(2.0) / (2.0 * db));
        uint32_t prev = 0xFFFFFFFFu;
        for (int64_t h = 1;; ++h) {
            const uint32_t v = to_u32_threshold(std::exp(-2.0 * (double)h * db));
            if (v == 0u) break;
            if (h > (1 << 22)) { *why = "exchange table longer than 2^22 entries (beta gap too small)"; return -1; }
            if (h > 1 && v > prev) { *why = "exchange table not monotone (host libm)"; return -1; }
            if (xthr) {
                if (n >= xcap) { *why = "exchange tables exceed the table capacity"; return -1; }
                xthr[n] = v;
            }
            prev = v;
            ++n;
        }
    }
    if (NT > 0) xoff[NT - 1] = n;
    return n;
}

// Returns an empty string or the reason the ladder is rejected.
inline std::string build_tables(int NT, int kt, const double* betas, Tables& tb)
{
    tb.kt = kt;
    tb.thr.assign((size_t)NT * kt, 0u);
    tb.xoff.assign((size_t)NT, 0);
    tb.xhint.assign((size_t)(NT > 1 ? NT - 1 : 1), 0.f);
    const char* why = "";
    const int64_t n = fill_tables(NT, kt, betas, tb.thr.data(), tb.xoff.data(), tb.xhint.data(), nullptr, 0, &why);
    if (n < 0) return why;
    if (n > (int64_t)INT32_MAX / 2) return "exchange tables too large";
    tb.xthr.assign((size_t)n, 0u);
    if (fill_tables(NT, kt, betas, tb.thr.data(), tb.xoff.data(), tb.xhint.data(), tb.xthr.data(), n, &why) < 0)
        return why;
    return "";
}

}  // namespace ptg
