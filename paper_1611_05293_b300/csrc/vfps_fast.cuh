// vfps_fast.cuh -- FP32 step kernel for grids with n a multiple of 4, written
// to issue few instructions per cell: rotation (2-D Lagrange, Sec. III.A-B),
// kick along p, Fokker-Planck step (Eq. cubic diff), column sums, and the
// same last-CTA finaliser as step_kernel.  The hot configuration (cubic
// interpolation, no clamp) is its own instance (NI = 4); N_I = 2 and 3 read
// the order from the descriptor (NI = 0: their nodes fit the cubic 4-slot
// layout with zero weights); clamping (Eq. clamping), at any order, is the
// NI = 1 instance: each interpolated value is restricted to its nearest
// nodes, which the same windows hold.
//
// Work of one lane: blocks of consecutive rows of its warp's column x.
//  * Rotation, four rows y0..y0+3.  Along a column the source point moves
//    by (-sin phi, ~1) cells per row, so the four outputs share one window
//    of 5 source columns x 12 rows, read with 15 LDS.128.  The y-node offset
//    floor(dy) is the same for all four rows and, almost always, for the
//    whole column (dy changes by cos phi - 1 ~ 1e-5 per row): the window's
//    row alignment is then uniform and selects a compile-time register
//    layout.  The x-node may step back by one inside the block (dx changes
//    by -sin phi per row); a 5-column weight vector with a zero at one end
//    covers both cases.  A column that does not meet these conditions is
//    computed cell by cell (rotate_cell_ring).
//  * Kick and Fokker-Planck, KR rows y0..y0+KR-1 (KR = 8, or 4 when n is
//    not a multiple of 8).  The column's kick shift s and weights are
//    uniform and come from a per-column table the finaliser of the previous
//    step wrote, with the pending renormalisation factor folded into the
//    weights; psi_b(y0-1..y0+KR+1) comes from one window of the psi_a column
//    (zero-padded rows), and psi_c(y0..y0+KR-1) from psi_b and the per-row
//    FP weights g_k(y), held as four planar rows in shared memory so that
//    the lanes' 16-byte reads do not conflict.
//  * Weight pairs of rows go through packed FP32x2 arithmetic (sm_100+).
#pragma once
#include "vfps_kernels.cuh"

namespace vfps {

constexpr int kColPad = 16;  // zero rows above and below each psi_a column

// Rotation passes (128 rows each) unrolled together in rotate_column.
#ifndef VFPS_ROT_UNROLL
#define VFPS_ROT_UNROLL 1
#endif
constexpr int kRotUnroll = VFPS_ROT_UNROLL;

// Row padding of the staged slab: covers the largest y-node offset plus the
// 12-row window, rounded to a multiple of 4 for 16-byte rows.
__host__ __device__ inline int fast_row_pad(int h) { return ((h + 4 + 3) / 4) * 4; }

// Pitch of a ring slot (rows -RP .. n+RP-1), rounded up to 32 floats: lanes
// of one warp that straddle two slots then still read distinct banks.
__host__ __device__ inline int ring_pitch(int n, int RP) { return (n + 2 * RP + 31) & ~31; }

// Pitch of a psi_a column (kColPad zero rows above, >= kColPad below),
// congruent to 32 floats modulo 64 (its half, in 16-byte chunks, is 4 mod 8).
__host__ __device__ inline int cola_pitch(int n) { return ((n + 63) & ~63) + 32; }

// Layout of the psi_a columns and FP-weight rows for 8-row kick blocks.  A
// lane of an 8-row block reads every other 16-byte chunk, which on a plain
// layout puts two lanes on each bank.  Chunk c of a row of HC2 chunks is
// therefore stored at c/2 + (c&1)*HC2/2: even chunks in the first half, odd
// ones in the second, so those reads hit consecutive chunks; lanes writing
// consecutive chunks alternate between halves that start 4 banks apart
// (psi_a columns, HC2/2 = 4 mod 8).  4-row blocks keep the plain layout.
template <int KR>
__device__ __forceinline__ int split_idx(int e, int half_chunks)
{
    if constexpr (KR == 8) {
        const int c = e >> 2;
        return (((c >> 1) + (c & 1) * half_chunks) << 2) | (e & 3);
    } else {
        return e;
    }
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Cubic Lagrange weights (nodes -1, 0, 1, 2) for two fractions at once.
// With m = t(1 - t) and k = 1 + m/2 the four cardinal polynomials are
//   w2 = t k,  w1 = (1 - t) k = k - w2,  w0 = m (t - 2)/6,  w3 = -m/2 - w0
// (w0 + w3 = -m/2 and w1 + w2 = k, so they sum to 1): seven operations.
// Each half of a pair is computed exactly as the scalar expression would be,
// so a broadcast pair (t, t) gives the weights of t in both halves.
__device__ __forceinline__ void lagrange2(float2 t, float2 w[4])
{
    const float2 m = __ffma2_rn(f2(-t.x, -t.y), t, t);                           // t - t^2
    const float2 k = __ffma2_rn(m, f2(0.5f, 0.5f), f2(1.f, 1.f));                // 1 + m/2
    w[2] = __fmul2_rn(t, k);
    w[1] = __fadd2_rn(k, f2(-w[2].x, -w[2].y));
    w[0] = __fmul2_rn(m, __ffma2_rn(t, f2(1.f / 6.f, 1.f / 6.f), f2(-1.f / 3.f, -1.f / 3.f)));
    w[3] = __ffma2_rn(m, f2(-0.5f, -0.5f), f2(-w[0].x, -w[0].y));
}

// lagrange2 for N_I nodes in the cubic 4-slot layout (lagrange_w4_rt): NI = 4
// is the compile-time cubic, NI = 0 and 1 take the order from ni; each half
// of a pair as the scalar weights are.
template <int NI>
__device__ __forceinline__ void lagrange2_ni(float2 t, float2 w[4], int ni)
{
    if constexpr (NI == 4) {
        lagrange2(t, w);
    } else {
        float a[4], b[4];
        lagrange_w4_rt(t.x, a, ni);
        lagrange_w4_rt(t.y, b, ni);
#pragma unroll
        for (int k = 0; k < 4; ++k) w[k] = f2(a[k], b[k]);
    }
}
template <int NI>
__device__ __forceinline__ void lagrange_w4(float t, float w[4], int ni)
{
    if constexpr (NI == 4) lagrange_w<float, 4>(t, w);
    else lagrange_w4_rt(t, w, ni);
}

// v restricted to [min(lo), max(hi)] of its nearest nodes (reading 4).
__device__ __forceinline__ float clamp_to(float v, float lo, float hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Fokker-Planck weight g_k(y) of tap k (rows y-1 .. y+2) with the identity
// folded into the centre tap, in one fixed order of operations (the FP32
// kernels all build their tables with it).
__device__ __forceinline__ float fp_weight(const Desc<float>& D, int k, int y)
{
    return (k == 1 ? 1.f : 0.f) + fmaf(D.gb[k], float(y), D.ga[k]);
}

// psi_c(y) = sum_k g_k(y) psi_b(y - 1 + k), in one fixed order.
__device__ __forceinline__ float fp_apply(float g0, float g1, float g2, float g3, const float* b)
{
    float v = g0 * b[0];
    v = fmaf(g1, b[1], v);
    v = fmaf(g2, b[2], v);
    return fmaf(g3, b[3], v);
}

// Rotation of four rows from a 5 x 12 register window: 5 consecutive slab
// columns (ring slots slot0.., row offset rowoff) whose first row is O rows
// above the first stencil row of output 0.  tx, ty hold the node fractions
// of rows (0,1) and (2,3) as pairs (packed weight arithmetic).
template <int O, int NI>
__device__ __forceinline__ void rotate_block(const float* __restrict__ ring, int slot0, int R, int P, int rowoff,
                                             float2 tx01, float2 tx23, float2 ty01, float2 ty23, bool e1,
                                             bool e2, bool e3, float out[4], int ni, bool clamp)
{
    // (NI = 1, clamped: the 2 x 2 nearest nodes of output k are window
    // columns 2 - e_k, 3 - e_k, rows O + k + 1, O + k + 2)
    float lo[4] = {3.4e38f, 3.4e38f, 3.4e38f, 3.4e38f}, hi[4] = {-3.4e38f, -3.4e38f, -3.4e38f, -3.4e38f};
    float2 wy01[4], wy23[4], wx01[4], wx23[4];
    lagrange2_ni<NI>(ty01, wy01, ni);
    lagrange2_ni<NI>(ty23, wy23, ni);
    lagrange2_ni<NI>(tx01, wx01, ni);
    lagrange2_ni<NI>(tx23, wx23, ni);
    const float wy[4][4] = {{wy01[0].x, wy01[1].x, wy01[2].x, wy01[3].x},
                            {wy01[0].y, wy01[1].y, wy01[2].y, wy01[3].y},
                            {wy23[0].x, wy23[1].x, wy23[2].x, wy23[3].x},
                            {wy23[0].y, wy23[1].y, wy23[2].y, wy23[3].y}};
    // x-weights over the 5 window columns: output k uses columns 1..4 when its
    // x-node equals row 0's, columns 0..3 when it stepped back by one
    const float wx[4][4] = {{wx01[0].x, wx01[1].x, wx01[2].x, wx01[3].x},
                            {wx01[0].y, wx01[1].y, wx01[2].y, wx01[3].y},
                            {wx23[0].x, wx23[1].x, wx23[2].x, wx23[3].x},
                            {wx23[0].y, wx23[1].y, wx23[2].y, wx23[3].y}};
    const bool e[4] = {false, e1, e2, e3};
    float2 acc01 = f2(0.f, 0.f), acc23 = f2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        const float4* cp = reinterpret_cast<const float4*>(ring + ((slot0 + a) & (R - 1)) * P + rowoff);
        const bool ok = VFPS_GUARD(rowoff >= 0 && rowoff + 12 <= P && slot0 >= 0 && slot0 < R, 2);
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 q0 = ok ? cp[0] : z4, q1 = ok ? cp[1] : z4, q2 = ok ? cp[2] : z4;
        const float win[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
        float r[4], wa[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float v = wy[k][0] * win[O + k];
            v = fmaf(wy[k][1], win[O + k + 1], v);
            v = fmaf(wy[k][2], win[O + k + 2], v);
            r[k] = fmaf(wy[k][3], win[O + k + 3], v);
            wa[k] = e[k] ? ((a <= 3) ? wx[k][a] : 0.f) : ((a >= 1) ? wx[k][a - 1] : 0.f);
            if constexpr (NI == 1) {
                if (clamp && (a == 2 - int(e[k]) || a == 3 - int(e[k]))) {
                    lo[k] = fminf(lo[k], fminf(win[O + k + 1], win[O + k + 2]));
                    hi[k] = fmaxf(hi[k], fmaxf(win[O + k + 1], win[O + k + 2]));
                }
            }
        }
        acc01 = __ffma2_rn(f2(wa[0], wa[1]), f2(r[0], r[1]), acc01);
        acc23 = __ffma2_rn(f2(wa[2], wa[3]), f2(r[2], r[3]), acc23);
    }
    out[0] = acc01.x;
    out[1] = acc01.y;
    out[2] = acc23.x;
    out[3] = acc23.y;
    if constexpr (NI == 1) {
        if (clamp)
#pragma unroll
            for (int k = 0; k < 4; ++k) out[k] = clamp_to(out[k], lo[k], hi[k]);
    }
}

// rotate_block when no row of the block steps back: the x-node of all four
// rows is row 0's, so only window columns 1..4 take part and the x-weights
// need no selection (same operations as rotate_block for such a block, whose
// column-0 terms are zeros).
template <int O, int NI>
__device__ __forceinline__ void rotate_block4(const float* __restrict__ ring, int slot0, int R, int P, int rowoff,
                                              float2 tx01, float2 tx23, float2 ty01, float2 ty23, float out[4], int ni,
                                              bool clamp)
{
    float lo[4] = {3.4e38f, 3.4e38f, 3.4e38f, 3.4e38f}, hi[4] = {-3.4e38f, -3.4e38f, -3.4e38f, -3.4e38f};
    float2 wy01[4], wy23[4], wx01[4], wx23[4];
    lagrange2_ni<NI>(ty01, wy01, ni);
    lagrange2_ni<NI>(ty23, wy23, ni);
    lagrange2_ni<NI>(tx01, wx01, ni);
    lagrange2_ni<NI>(tx23, wx23, ni);
    float2 acc01, acc23;
#pragma unroll
    for (int a = 1; a < 5; ++a) {
        const float4* cp = reinterpret_cast<const float4*>(ring + ((slot0 + a) & (R - 1)) * P + rowoff);
        const bool ok = VFPS_GUARD(rowoff >= 0 && rowoff + 12 <= P && slot0 >= 0 && slot0 < R, 2);
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 q0 = ok ? cp[0] : z4, q1 = ok ? cp[1] : z4, q2 = ok ? cp[2] : z4;
        const float win[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
        // rows (0, 1) and (2, 3) as packed pairs: the same operations per row
        float2 r01 = __fmul2_rn(wy01[0], f2(win[O], win[O + 1]));
        float2 r23 = __fmul2_rn(wy23[0], f2(win[O + 2], win[O + 3]));
#pragma unroll
        for (int b = 1; b < 4; ++b) {
            r01 = __ffma2_rn(wy01[b], f2(win[O + b], win[O + b + 1]), r01);
            r23 = __ffma2_rn(wy23[b], f2(win[O + b + 2], win[O + b + 3]), r23);
        }
        const float r[4] = {r01.x, r01.y, r23.x, r23.y};
        if constexpr (NI == 1) {
            if (clamp && (a == 2 || a == 3))
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    lo[k] = fminf(lo[k], fminf(win[O + k + 1], win[O + k + 2]));
                    hi[k] = fmaxf(hi[k], fmaxf(win[O + k + 1], win[O + k + 2]));
                }
        }
        if (a == 1) {
            acc01 = __fmul2_rn(wx01[0], f2(r[0], r[1]));
            acc23 = __fmul2_rn(wx23[0], f2(r[2], r[3]));
        } else {
            acc01 = __ffma2_rn(wx01[a - 1], f2(r[0], r[1]), acc01);
            acc23 = __ffma2_rn(wx23[a - 1], f2(r[2], r[3]), acc23);
        }
    }
    out[0] = acc01.x;
    out[1] = acc01.y;
    out[2] = acc23.x;
    out[3] = acc23.y;
    if constexpr (NI == 1) {
        if (clamp)
#pragma unroll
            for (int k = 0; k < 4; ++k) out[k] = clamp_to(out[k], lo[k], hi[k]);
    }
}

// Offset of the psi_a column row kColPad + yb + 4 lane (start of a
// lane's 4-row rotation block, yb a multiple of 128) in the column layout:
// the lane part, to which 2 (kColPad/4 + yb/4) (split layout) or kColPad + yb
// (plain layout) is added.
template <int KR>
__device__ __forceinline__ int cola_lane_base(int lane, int HC)
{
    if constexpr (KR == 8) return ((lane >> 1) + (lane & 1) * HC) << 2;
    else return 4 * lane;
}
template <int KR>
__device__ __forceinline__ int cola_block_off(int yb)
{
    if constexpr (KR == 8) return 2 * ((kColPad >> 2) + (yb >> 2));
    else return kColPad + yb;
}

// Kick + Fokker-Planck for the lane's blocks of KR rows of one column.  The
// psi_a window starts O2 rows above the first row the kick of row y0-1
// needs (A2 = s - 2 + kColPad: column index of row y0+s-2, minus y0; PAR =
// parity of its 16-byte chunk, fixed per column for 8-row blocks); w are the
// column's kick weights (pending scale included), s its node shift; g holds
// the FP weights g_k(y) as four rows of n (split layout for KR = 8), with
// the identity folded into the centre tap: psi_c(y) = sum_k g_k(y) psi_b(y-1+k).
// Rows ylo .. yhi - 1 (block-aligned: multiples of 32 KR, yhi = n or such a
// multiple).  SMALL: s is -1 or 0 (kicks under one cell), where the edge test
// reduces to the rows just outside the grid.  NI = 1 (clamped): each psi_b value is
// restricted to its two nearest nodes (times csf).
//
// FP = false (the RF kick of the Manhattan rotation): only the shift, psi_b of
// the lane's own rows goes to the psi_a-layout column dst (shared memory).
template <int O2, int PAR, int KR, bool SMALL, bool FP = true, int NI = 4>
__device__ __forceinline__ float kick_fp_column(const float* __restrict__ colcol, int HC,
                                                const float* __restrict__ g, float* __restrict__ dst, int n, int s,
                                                int A2, float4 w, int lane, bool clamp, float csf, int ylo, int yhi)
{
    constexpr int NB = KR + 3;                  // psi_b rows y0-1 .. y0+KR+1
    constexpr int NV = (O2 + NB + 3 + 3) / 4;   // float4 reads of the window
    // psi_b(y) is 0 off the grid and where its source is > 1 cell outside
    const int lo = max(0, -1 - s), hi = min(n - 1, n - 1 - s);
    float lsum = 0.f;
#pragma unroll
    for (int yb = ylo; yb < yhi; yb += 32 * KR) {
        const int y0 = yb + KR * lane;
        if ((n % (32 * KR)) && y0 >= n) break;
        float win[4 * NV];
        // window rows y0 + A2 - O2 .. + 4 NV - 1 of the padded column (8 HC rows)
        const bool wok = VFPS_GUARD(y0 + A2 - O2 >= 0 && y0 + A2 - O2 + 4 * NV <= 8 * HC, 4);
        if (!wok) {
#pragma unroll
            for (int v = 0; v < 4 * NV; ++v) win[v] = 0.f;
        } else if constexpr (KR == 8) {
            // chunk of window row 4v: (y0 + A2 - O2)/4 + v = 2*(y0/8 + m) + PAR + v
            const float* b0 = colcol + 4 * ((y0 >> 3) + ((A2 >> 2) >> 1));
            const float* b1 = b0 + 4 * HC;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float4 q = *reinterpret_cast<const float4*>(((PAR + v) & 1 ? b1 : b0) + 4 * ((PAR + v) >> 1));
                win[4 * v] = q.x;
                win[4 * v + 1] = q.y;
                win[4 * v + 2] = q.z;
                win[4 * v + 3] = q.w;
            }
        } else {
            const float4* wp = reinterpret_cast<const float4*>(colcol + y0 + A2 - O2);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float4 q = wp[v];
                win[4 * v] = q.x;
                win[4 * v + 1] = q.y;
                win[4 * v + 2] = q.z;
                win[4 * v + 3] = q.w;
            }
        }
        // psi_b(y0 + j - 1): nodes y0+j+s-2 .. y0+j+s+1
        float b[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            float v = w.x * win[O2 + j];
            v = fmaf(w.y, win[O2 + j + 1], v);
            v = fmaf(w.z, win[O2 + j + 2], v);
            b[j] = fmaf(w.w, win[O2 + j + 3], v);
        }
        if constexpr (NI == 1) {
            // clamped: between its two nearest nodes, window rows O2 + j + 1, + 2
            // (times csf, the pending scale that the weights carry)
            if (clamp)
#pragma unroll
                for (int j = 0; j < NB; ++j)
                    b[j] = clamp_to(b[j], csf * fminf(win[O2 + j + 1], win[O2 + j + 2]),
                                    csf * fmaxf(win[O2 + j + 1], win[O2 + j + 2]));
        }
        if constexpr (SMALL) {
            // s in {-1, 0}: every on-grid row has its source within one cell
            // of the grid, so only the rows -1, n, n+1 are zeroed
            if (y0 == 0) b[0] = 0.f;
            if (y0 + KR == n) {
                b[NB - 2] = 0.f;
                b[NB - 1] = 0.f;
            }
        } else {
            const int jlo = lo - y0 + 1, jhi = hi - y0 + 1;
#pragma unroll
            for (int j = 0; j < NB; ++j) b[j] = (j >= jlo && j <= jhi) ? b[j] : 0.f;
        }
        if constexpr (!FP) {
#pragma unroll
            for (int q4 = 0; q4 < KR / 4; ++q4)
                if (VFPS_GUARD(kColPad + y0 + 4 * q4 + 4 <= 8 * HC, 5))
                    *reinterpret_cast<float4*>(dst + split_idx<KR>(kColPad + y0 + 4 * q4, HC)) =
                        make_float4(b[4 * q4 + 1], b[4 * q4 + 2], b[4 * q4 + 3], b[4 * q4 + 4]);
        } else {
#pragma unroll
        for (int q4 = 0; q4 < KR / 4; ++q4) {
            const int y = y0 + 4 * q4;
            const int gi = (KR == 8) ? 4 * (y0 >> 3) + q4 * (n >> 1) : y;  // split_idx<KR>(y, n/8)
            const float4 g0 = *reinterpret_cast<const float4*>(g + gi);
            const float4 g1 = *reinterpret_cast<const float4*>(g + n + gi);
            const float4 g2 = *reinterpret_cast<const float4*>(g + 2 * n + gi);
            const float4 g3 = *reinterpret_cast<const float4*>(g + 3 * n + gi);
            const float ga[4] = {g0.x, g0.y, g0.z, g0.w}, gb[4] = {g1.x, g1.y, g1.z, g1.w};
            const float gc[4] = {g2.x, g2.y, g2.z, g2.w}, gd[4] = {g3.x, g3.y, g3.z, g3.w};
            float c[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) c[k] = fp_apply(ga[k], gb[k], gc[k], gd[k], b + 4 * q4 + k);
            *reinterpret_cast<float4*>(dst + y) = make_float4(c[0], c[1], c[2], c[3]);
            lsum += (c[0] + c[1]) + (c[2] + c[3]);
        }
        }
    }
    return lsum;
}

// Source node (mx, my) and cubic weights of cell (x, y) of the rotation, in
// one fixed order of operations; false when the source lies more than one
// cell outside the grid (the cell is then 0).
template <int NI>
__device__ __forceinline__ bool cell_weights(int x, int y, int n, float cm1, float sn, float c, int* mx, int* my,
                                             float wx[4], float wy[4], int ni)
{
    const float xc = float(x) - c, yc = float(y) - c;
    const float dx = fmaf(-sn, yc, cm1 * xc);
    const float dy = fmaf(cm1, yc, sn * xc);
    const float fx = floorf(dx), fy = floorf(dy);
    *mx = x + int(fx);
    *my = y + int(fy);
    if (*mx <= -2 || *mx >= n || *my <= -2 || *my >= n) return false;
    lagrange_w4<NI>(dx - fx, wx, ni);
    lagrange_w4<NI>(dy - fy, wy, ni);
    return true;
}

// Rotation of one cell from the column ring (general path), with slab
// column col stored in ring slot col & (R-1).
template <int NI>
__device__ __forceinline__ float rotate_cell_ring(const float* __restrict__ ring, int R, int P, int RP, int x, int y,
                                                  int n, float cm1, float sn, float c, int ni, bool clamp)
{
    int mx, my;
    float wx[4], wy[4];
    if (!cell_weights<NI>(x, y, n, cm1, sn, c, &mx, &my, wx, wy, ni)) return 0.f;
    float acc = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const float* col = ring + ((mx - 1 + a) & (R - 1)) * P + (my - 1 + RP);
        float r = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) r = fmaf(wy[b], col[b], r);
        acc = fmaf(wx[a], r, acc);
    }
    if constexpr (NI == 1) {
        if (clamp) {  // the 2 x 2 nearest nodes (mx, my) .. (mx + 1, my + 1)
            const float* c0 = ring + (mx & (R - 1)) * P + my + RP;
            const float* c1 = ring + ((mx + 1) & (R - 1)) * P + my + RP;
            acc = clamp_to(acc, fminf(fminf(c0[0], c0[1]), fminf(c1[0], c1[1])),
                           fmaxf(fmaxf(c0[0], c0[1]), fmaxf(c1[0], c1[1])));
        }
    }
    return acc;
}

// Issue cp.async copies of slab columns col0 .. col0+ncols-1 into their ring
// slots: rows 0 .. n-1 only (the RP padding rows above and below stay zero
// from the CTA's start); columns outside the grid are zero-filled.  Warp w
// takes columns col0+w, col0+w+W, ...
template <int W>
__device__ __forceinline__ void load_columns(float* ring, int R, int P, int RP, const float* __restrict__ in,
                                             int ld, int n, int col0, int ncols)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n4 = n >> 2;
    for (int k = warp; k < ncols; k += W) {
        const int gx = col0 + k;
        float* dst = ring + (size_t)(gx & (R - 1)) * P + RP + 4 * lane;
        if (!VFPS_GUARD(RP + n <= P, 1)) continue;
        if (gx >= 0 && gx < n) {
            const float* src = in + (size_t)gx * ld + 4 * lane;
            for (int r4 = lane; r4 < n4; r4 += 32, dst += 128, src += 128) cp_async16(dst, src, 16);
        } else {
            for (int r4 = lane; r4 < n4; r4 += 32, dst += 128)
                *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

__host__ __device__ inline int ring_slots(int W, int h)
{
    int r = 1;
    while (r < 2 * W + 2 * h) r <<= 1;
    return r;
}

// Shared memory of the FP32 streaming kernel: ring, psi_a columns, FP
// weights, a 4-stage buffer of the tiles' kick-table entries, for the
// Manhattan rotation a second set of columns (the RF-kicked psi), and for
// n >= 512 the upper-half lane partials of the W columns.
__host__ inline size_t fast_ring_smem(int n, int h, int W, bool manhattan)
{
    const int RP = fast_row_pad(h);
    return (size_t)ring_slots(W, h) * ring_pitch(n, RP) * 4 + (size_t)W * cola_pitch(n) * 4 * (manhattan ? 2 : 1) +
           (size_t)n * 16 + (size_t)4 * W * 32 + (n >= 512 ? (size_t)W * 32 * 4 : 0);
}

// Copy the kick-table entries (two float4) of column x into dst (lanes 0 and
// 1 of the calling warp); columns past the grid get zeros.
__device__ __forceinline__ void load_kick(float4* dst, const float4* __restrict__ kickw, int x, int n, int lane)
{
    if (lane < 2) {
        const bool ok = x < n;
        cp_async16(dst + lane, ok ? kickw + 2 * x + lane : kickw, ok ? 16 : 0);
    }
}

// Rotation of one column x (rows ylo..yhi-1, four per lane and pass) when the
// y-node offset FY is the same on every row (window alignment O = A & 3,
// A = FY - 1 + RP) and the x-node steps back by at most one inside a block
// of four rows (sin phi < 1/3).
template <int O, int KR, int NI>
__device__ __forceinline__ void rotate_column(const float* __restrict__ ring, int R, int P, int RP, int A,
                                              float* __restrict__ colcol, int HC, int x, int n, int lane, float xc,
                                              float c, float sn, float cm1, int FY, int ni, bool clamp, int ylo,
                                              int yhi)
{
    const float2 msn2 = f2(-sn, -sn), cm12 = f2(cm1, cm1);
    const float2 snxc = f2(sn * xc, sn * xc), cmxc = f2(cm1 * xc, cm1 * xc);
    const float fyf = float(FY);
    const float2 mfy = f2(-fyf, -fyf);
    const int lbase = cola_lane_base<KR>(lane, HC);
#pragma unroll kRotUnroll
    for (int yb = ylo; yb < yhi; yb += 128) {
        // every lane runs every pass (the vote below needs the whole warp);
        // lanes past the last row only vote
        const int y0 = yb + 4 * lane;
        const bool live = !(n & 127) || y0 < n;
        const float yc0 = float(y0) - c;
        const float2 yc01 = f2(yc0, yc0 + 1.f), yc23 = f2(yc0 + 2.f, yc0 + 3.f);
        // dx = (cos phi - 1) xc - sin phi yc,  dy = sin phi xc + (cos phi - 1) yc
        const float2 dx01 = __ffma2_rn(msn2, yc01, cmxc);
        const float2 dx23 = __ffma2_rn(msn2, yc23, cmxc);
        const float2 ty01 = __fadd2_rn(__ffma2_rn(cm12, yc01, snxc), mfy);
        const float2 ty23 = __fadd2_rn(__ffma2_rn(cm12, yc23, snxc), mfy);
        const float fx0 = floorf(dx01.x), fx1 = floorf(dx01.y), fx2 = floorf(dx23.x), fx3 = floorf(dx23.y);
        const float2 tx01 = f2(dx01.x - fx0, dx01.y - fx1), tx23 = f2(dx23.x - fx2, dx23.y - fx3);
        const int mx0 = x + int(fx0);
        float r[4];
        // the x-node steps back inside the block iff it does at row 3; most
        // passes have no such block in the whole warp and skip window column 0
        const bool anyback = __any_sync(0xffffffffu, live && fx3 < fx0);
        if (!live) continue;
        if (anyback)
            rotate_block<O, NI>(ring, (mx0 - 2) & (R - 1), R, P, y0 + A - O, tx01, tx23, ty01, ty23, fx1 < fx0,
                                fx2 < fx0, fx3 < fx0, r, ni, clamp);
        else
            rotate_block4<O, NI>(ring, (mx0 - 2) & (R - 1), R, P, y0 + A - O, tx01, tx23, ty01, ty23, r, ni, clamp);
        // sources more than one cell outside the grid give 0
        if (!((mx0 >= 0) && (mx0 <= n - 1) && (y0 + FY >= -1) && (y0 + 3 + FY <= n - 1))) {
            const float fxk[4] = {fx0, fx1, fx2, fx3};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int mx = x + int(fxk[k]), my = y0 + k + FY;
                if (mx <= -2 || mx >= n || my <= -2 || my >= n) r[k] = 0.f;
            }
        }
        if (VFPS_GUARD(kColPad + y0 + 4 <= 8 * HC, 5))
            *reinterpret_cast<float4*>(colcol + lbase + cola_block_off<KR>(yb)) = make_float4(r[0], r[1], r[2], r[3]);
    }
}

// Manhattan rotation, first half (Sec. III.B, symplectic rotation): the drift
// q -> q + h p moves row y along q by h (y - c) cells, psi_a(x, y) = psi(x -
// h (y - c), y), interpolated along q (cubic).  Four rows y0..y0+3 per lane
// and pass; their x-node steps down by at most one inside the block (h <
// 1/3), so one 5-column window of the ring (one LDS.128 per column) with a
// 5-column weight vector covers the block, as in the 2-D rotation.
template <int KR, int NI>
__device__ __forceinline__ void drift_column(const float* __restrict__ ring, int R, int P, int RP,
                                             float* __restrict__ colcol, int HC, int x, int n, int lane, float c,
                                             float hm, int ni, bool clamp, int ylo, int yhi)
{
    const int lbase = cola_lane_base<KR>(lane, HC);
#pragma unroll 1
    for (int yb = ylo; yb < yhi; yb += 128) {
        const int y0 = yb + 4 * lane;
        if ((n & 127) && y0 >= n) break;
        const float yc0 = float(y0) - c;
        const float d0 = -hm * yc0, d1 = -hm * (yc0 + 1.f), d2 = -hm * (yc0 + 2.f), d3 = -hm * (yc0 + 3.f);
        const float fx0 = floorf(d0), fx1 = floorf(d1), fx2 = floorf(d2), fx3 = floorf(d3);
        float2 w01[4], w23[4];
        lagrange2_ni<NI>(f2(d0 - fx0, d1 - fx1), w01, ni);
        lagrange2_ni<NI>(f2(d2 - fx2, d3 - fx3), w23, ni);
        const float wx[4][4] = {{w01[0].x, w01[1].x, w01[2].x, w01[3].x},
                                {w01[0].y, w01[1].y, w01[2].y, w01[3].y},
                                {w23[0].x, w23[1].x, w23[2].x, w23[3].x},
                                {w23[0].y, w23[1].y, w23[2].y, w23[3].y}};
        const bool e[4] = {false, fx1 < fx0, fx2 < fx0, fx3 < fx0};
        const int mx0 = x + int(fx0);
        const int slot0 = (mx0 - 2) & (R - 1);  // window columns mx0-2 .. mx0+2
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        float lo[4] = {3.4e38f, 3.4e38f, 3.4e38f, 3.4e38f}, hi[4] = {-3.4e38f, -3.4e38f, -3.4e38f, -3.4e38f};
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            const float4 q = VFPS_GUARD(RP + y0 + 4 <= P && slot0 >= 0 && slot0 < R, 3)
                                 ? *reinterpret_cast<const float4*>(ring + ((slot0 + a) & (R - 1)) * P + RP + y0)
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            const float v[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float wa = e[k] ? ((a <= 3) ? wx[k][a] : 0.f) : ((a >= 1) ? wx[k][a - 1] : 0.f);
                acc[k] = fmaf(wa, v[k], acc[k]);
                if constexpr (NI == 1) {  // nearest nodes: window columns 2 - e_k, 3 - e_k
                    if (clamp && (a == 2 - int(e[k]) || a == 3 - int(e[k]))) {
                        lo[k] = fminf(lo[k], v[k]);
                        hi[k] = fmaxf(hi[k], v[k]);
                    }
                }
            }
        }
        if constexpr (NI == 1) {
            if (clamp)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[k] = clamp_to(acc[k], lo[k], hi[k]);
        }
        // sources more than one cell outside the grid give 0
        if (!(mx0 >= 0 && mx0 <= n - 1)) {
            const float fxk[4] = {fx0, fx1, fx2, fx3};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int mx = x + int(fxk[k]);
                if (mx <= -2 || mx >= n) acc[k] = 0.f;
            }
        }
        if (VFPS_GUARD(kColPad + y0 + 4 <= 8 * HC, 5))
            *reinterpret_cast<float4*>(colcol + lbase + cola_block_off<KR>(yb)) =
                make_float4(acc[0], acc[1], acc[2], acc[3]);
    }
}

// Moment-recording steps only: for the ncols columns from xs that this CTA
// has just written to out, sum_y p_y psi_c(y) and sum_y p_y^2 psi_c(y) into
// D.colmom[2x], [2x+1] (p_y = (y - c) Delta).  FP32 within a column (lane
// partials, then across lanes -- on this GPU's FP64 pipe, two FP64 shuffle
// trees per column cost more than the pass itself), FP64 across columns in
// the finaliser.  Warp w takes columns xs+w, xs+w+W, ...
__device__ __noinline__ void strip_p_moments(const Desc<float>& D, const float* out, int xs, int ncols, int n, int ld)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const float dl = float(D.delta), cc = D.c;
    for (int k = warp; k < ncols && xs + k < n; k += nw) {
        const int x = xs + k;
        const float* col = out + (size_t)x * ld;
        float a1 = 0.f, a2 = 0.f;
        for (int y = lane; y < n; y += 32) {
            const float p = (float(y) - cc) * dl, pv = p * col[y];
            a1 += pv;
            a2 = fmaf(p, pv, a2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a1 += __shfl_down_sync(0xffffffffu, a1, o);
            a2 += __shfl_down_sync(0xffffffffu, a2, o);
        }
        if (lane == 0) {
            D.colmom[2 * x] = double(a1);
            D.colmom[2 * x + 1] = double(a2);
        }
    }
}

// ----------------------------------------------------------------------------
// Persistent launches (one lone simulation, K steps per launch; see
// step_persistent_f32 for the protocol).
struct PersistStep {
    int k;          // step of this launch, 0 .. K-1
    int par;        // psi[par] holds the state this step reads
    long long t;    // steps done before this one
};

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_s32(const int* p)
{
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// One poll step of a bounded wait: false once the wait has to give up (the
// poll count reached D.spin_limit, or another CTA gave up: status
// VFPS_ETIMEOUT, checked every 64 polls), after setting that status.  No
// sleep between polls: each poll is a dependent L2 load, which paces the
// loop (a sleeping poller noticed a new value microseconds late).
#ifndef VFPS_POLL_NS
#define VFPS_POLL_NS 0
#endif
__device__ __forceinline__ bool poll_on(const Desc<float>& D, unsigned& polls)
{
    ++polls;
    if (polls >= D.spin_limit || ((polls & 63) == 0 && ld_volatile_s32(&D.st->status) == -4)) {
        atomicExch(&D.st->status, -4);
        return false;
    }
    if (VFPS_POLL_NS > 0) __nanosleep(VFPS_POLL_NS);
    return true;
}

// Bounded wait of one thread for the tagged words p[0 .. NW-1] of launch
// step tag (loaded together each poll); their values go to out.
template <int NW>
__device__ __forceinline__ bool wait_tagged(const Desc<float>& D, const unsigned long long* p, unsigned tag,
                                            unsigned* out)
{
    unsigned polls = 0;
    for (;;) {
        unsigned long long w[NW];
        bool all = true;
#pragma unroll
        for (int i = 0; i < NW; ++i) w[i] = ld_tagged(p + i);
#pragma unroll
        for (int i = 0; i < NW; ++i) all = all && (unsigned)(w[i] >> 32) == tag;
        if (all) {
#pragma unroll
            for (int i = 0; i < NW; ++i) out[i] = (unsigned)w[i];
            return true;
        }
        if (!poll_on(D, polls)) return false;
    }
}

// Bounded wait of a whole CTA until the step flags D.cflag[c0 .. c1] are all
// >= target (thread i polls flag c0 + i with relaxed loads, sleeping between
// polls, then fences: acquire).  A thread gives up after D.spin_limit polls,
// or as soon as another CTA has given up (status VFPS_ETIMEOUT, checked
// every 64 polls), after setting that status.  Every thread gets the
// outcome; after a true result the writes that preceded the matching flag
// releases are visible to all threads of the CTA.
__device__ __forceinline__ bool cta_wait_flags(const Desc<float>& D, int c0, int c1, unsigned target, int* s_ok)
{
    if (threadIdx.x == 0) *s_ok = 1;
    __syncthreads();
    for (int c = c0 + (int)threadIdx.x; c <= c1; c += blockDim.x) {
        unsigned polls = 0;
        bool ok = true;
        while (ld_relaxed_u32(D.cflag + c) < target)
            if (!(ok = poll_on(D, polls))) break;
        if (!ok) {
            *s_ok = 0;
            break;
        }
        fence_acq_rel_gpu();
    }
    __syncthreads();
    return *s_ok != 0;
}

// One strip of the streaming FP32 step: T consecutive W-column tiles of
// simulation D from column xs.  The strip walks its tiles one by one.  The
// slab columns live in a ring of R shared-memory slots (R >= 2W + 2h): while
// tile j is computed, the W new columns of tile j+1 are resident or landing
// and those of tile j+2 are requested, so each column of psi is read from
// HBM once per strip and the copies overlap the arithmetic.  psi_a stays
// unscaled; the pending renormalisation factor is part of the kick weights.
// The column sums of a strip are made visible with one fence per thread
// before the CTA takes the simulation's ticket; the CTA that takes the last
// ticket runs the finaliser.
//
// PERSIST (step ps->k of a persistent launch): the parity and step count come
// from ps; the shared-memory prologue (zero padding, FP weights) runs on the
// launch's first step only.  From the launch's second step on, the kick of a
// column is not in the table yet when the strip starts: after rotating a
// column, its warp waits for the column's kick record and the CTA's scale
// word (lanes 0 and 1, bounded) and builds the kick entry from them (kick_entry, as the finaliser does for the
// table).  Column sums go out as tagged words the finaliser CTA polls; at
// the end the CTA sets its step flag instead of taking a ticket.
// s_last is then the CTA's failure flag.  Returns false when a wait ran out
// (status set).
template <int W, int KR, int NC, int ROT, bool PERSIST = false, int NI = 4, int RS = (NC >= 512 ? 2 : 1)>
__device__ __forceinline__ bool strip_f32(const Desc<float>& D, int xs, int T, unsigned char* smem, int& s_last,
                                          const PersistStep* ps = nullptr)
{
    // NC > 0: the grid size is a compile-time constant (the hot sizes), so
    // loop bounds and pitches fold into the code; ld = n for FP32 then
    const int n = NC ? NC : D.n, ld = NC ? NC : D.ld, h = D.h;
    const int RP = fast_row_pad(h);
    const int P = ring_pitch(n, RP);
    const int R = ring_slots(W, h);
    const int PA = cola_pitch(n);
    const int HC = PA / 8;  // chunks in half a psi_a column (split layout)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float cm1 = D.cm1, sn = D.sn, c = D.c;
    const float4* __restrict__ kickw = D.kickw;
    double* __restrict__ colsum = D.colsum;
    // Rows of a column: in two halves split at Y2 where n >= 512 (its column
    // sum is then the lower half's lane partials plus the upper half's, for
    // every kernel shape); with RS = 2 (the N = 512 and 1024 instances) two
    // warps share a column, warp w taking column w % W, half w / W, so that
    // twice as many warps are resident at the same shared memory.
    constexpr int NW = W * RS;
    const int Y2 = n >= 512 ? ((n >> 1) & ~255) : n;
    const int cw = RS == 2 ? warp % W : warp, half = RS == 2 ? warp / W : 0;
    const int ylo = half ? Y2 : 0, yhi = (RS == 2 && !half) ? Y2 : n;

    float* ring = reinterpret_cast<float*>(smem);
    float* colA = ring + R * P;
    float* gtab = colA + W * PA;  // g_0(y) .. g_3(y), n each (split layout for KR = 8)
    float* colcol = colA + cw * PA;  // this warp's psi_a column, padded
    float4* kbuf = reinterpret_cast<float4*>(gtab + 4 * n) + 2 * cw;  // stage k: kbuf + 2 W k
    constexpr int rot = ROT;            // 1: Manhattan rotation (every instance of the launch)
    const float hm = D.hm;
    const int ni = NI == 4 ? 4 : D.ni;  // interpolation points (NI = 0: from the descriptor)
    const bool clamp = NI == 1;  // clamped interpolation (the NI = 1 instance)
    float* colbcol = reinterpret_cast<float*>(reinterpret_cast<float4*>(gtab + 4 * n) + 8 * W) + cw * PA;
    // RS = 2: the upper half's lane partials of each column
    float* xsum = reinterpret_cast<float*>(reinterpret_cast<float4*>(gtab + 4 * n) + 8 * W) + (rot ? W * PA : 0);

    // padding rows of every ring slot and of this warp's psi_a column: zero
    // for the whole strip (a persistent launch: for all its steps)
    if (!PERSIST || ps->k == 0) {
    for (int slot = warp; slot < R; slot += NW)
        for (int r = lane; r < RP; r += 32) {
            ring[slot * P + r] = 0.f;
            ring[slot * P + RP + n + r] = 0.f;
        }
    if (half == 0)
        for (int r = lane; r < PA - n; r += 32) colcol[split_idx<KR>(r < kColPad ? r : n + r, HC)] = 0.f;
    if (rot && half == 0)
        for (int r = lane; r < PA - n; r += 32) colbcol[split_idx<KR>(r < kColPad ? r : n + r, HC)] = 0.f;
    for (int y = threadIdx.x; y < n; y += blockDim.x) {
        const int gi = split_idx<KR>(y, n >> 3);
#pragma unroll
        for (int k = 0; k < 4; ++k) gtab[k * n + gi] = fp_weight(D, k, y);
    }
    }
    // what the previous step wrote (state word, psi, kick table) is read from here on
    if constexpr (!PERSIST) pdl_wait();
    const int par = PERSIST ? ps->par : D.st->parity;
    // kicks from the tagged records (persistent launch, not its first step)
    const bool recs = PERSIST && ps->k > 0;
    if (PERSIST && threadIdx.x == 0) s_last = 0;
    const float* __restrict__ in = D.psi[par];
    float* __restrict__ out = D.psi[par ^ 1];
    // a moment-recording step (the finaliser also needs each column's p-moments)
    const long long t_step = PERSIST ? ps->t : D.st->t;
    const bool mom_now = D.mom_every > 0 && (t_step + 1) % D.mom_every == 0;
    // window of tile 0, then the new columns of tile 1
    load_columns<NW>(ring, R, P, RP, in, ld, n, xs - h, W + 2 * h);
    if (!recs && half == 0) load_kick(kbuf, kickw, xs + cw, n, lane);
    cp_async_commit();
    if (T > 1) {
        load_columns<NW>(ring, R, P, RP, in, ld, n, xs + W + h, W);
        if (!recs && half == 0) load_kick(kbuf + 2 * W, kickw, xs + W + cw, n, lane);
    }
    cp_async_commit();

    for (int j = 0; j < T; ++j) {
        const int x = xs + j * W + cw;
        const bool active = x < n;
        cp_async_wait_1();
        __syncthreads();
        if (active && rot) {
            drift_column<KR, NI>(ring, R, P, RP, colcol, HC, x, n, lane, c, hm, ni, clamp, ylo, yhi);
        } else if (active) {
            const float xc = float(x) - c;
            // dy is linear along the column: floor(dy) is the same on every row
            // iff it is at the first and the last row
            const float fy_top = floorf(fmaf(cm1, 0.f - c, sn * xc));
            const float fy_bot = floorf(fmaf(cm1, float(n - 1) - c, sn * xc));
            if (fy_top == fy_bot && sn < 0.3f) {
                const int FY = int(fy_top);
                const int A = FY - 1 + RP;
                switch (A & 3) {
                case 0: rotate_column<0, KR, NI>(ring, R, P, RP, A, colcol, HC, x, n, lane, xc, c, sn, cm1, FY, ni, clamp, ylo, yhi); break;
                case 1: rotate_column<1, KR, NI>(ring, R, P, RP, A, colcol, HC, x, n, lane, xc, c, sn, cm1, FY, ni, clamp, ylo, yhi); break;
                case 2: rotate_column<2, KR, NI>(ring, R, P, RP, A, colcol, HC, x, n, lane, xc, c, sn, cm1, FY, ni, clamp, ylo, yhi); break;
                default: rotate_column<3, KR, NI>(ring, R, P, RP, A, colcol, HC, x, n, lane, xc, c, sn, cm1, FY, ni, clamp, ylo, yhi); break;
                }
            } else {
                for (int y = ylo + lane; y < yhi; y += 32)
                    colcol[split_idx<KR>(kColPad + y, HC)] = rotate_cell_ring<NI>(ring, R, P, RP, x, y, n, cm1, sn, c, ni, clamp);
            }
        }
        if constexpr (RS == 2) __syncthreads();  // both halves of every psi_a column
        else __syncwarp();
        const float* kcol = colcol;  // the column the wake kick reads
        if (active && rot) {
            // Manhattan rotation, second half: RF kick p -> p - h q, i.e. this
            // column moves along p by h (x - c) cells (source y + h (x - c))
            const float ts = hm * (float(x) - c), fk = floorf(ts);
            const int sr = int(fk);
            float wr[4];
            lagrange_w4<NI>(ts - fk, wr, ni);
            const float4 w4 = make_float4(wr[0], wr[1], wr[2], wr[3]);
            if (sr >= -4 && sr <= 4) {
                const int A2 = sr - 2 + kColPad;
                switch (KR == 8 ? (A2 & 7) : (A2 & 3)) {
                case 0: kick_fp_column<0, 0, KR, false, false, NI>(colcol, HC, gtab, colbcol, n, sr, A2, w4, lane, clamp, 1.f, ylo, yhi); break;
                case 1: kick_fp_column<1, 0, KR, false, false, NI>(colcol, HC, gtab, colbcol, n, sr, A2, w4, lane, clamp, 1.f, ylo, yhi); break;
                case 2: kick_fp_column<2, 0, KR, false, false, NI>(colcol, HC, gtab, colbcol, n, sr, A2, w4, lane, clamp, 1.f, ylo, yhi); break;
                case 3: kick_fp_column<3, 0, KR, false, false, NI>(colcol, HC, gtab, colbcol, n, sr, A2, w4, lane, clamp, 1.f, ylo, yhi); break;
                case 4: kick_fp_column<0, 1, KR, false, false, NI>(colcol, HC, gtab, colbcol, n, sr, A2, w4, lane, clamp, 1.f, ylo, yhi); break;
                case 5: kick_fp_column<1, 1, KR, KR == 8, false, NI>(colcol, HC, gtab, colbcol, n, sr, A2, w4, lane, clamp, 1.f, ylo, yhi); break;
                case 6: kick_fp_column<2, 1, KR, KR == 8, false, NI>(colcol, HC, gtab, colbcol, n, sr, A2, w4, lane, clamp, 1.f, ylo, yhi); break;
                default: kick_fp_column<3, 1, KR, false, false, NI>(colcol, HC, gtab, colbcol, n, sr, A2, w4, lane, clamp, 1.f, ylo, yhi); break;
                }
            } else {
                for (int y = ylo + lane; y < yhi; y += 32) {
                    const int m = y + sr;
                    float v = 0.f;
                    if (m > -2 && m < n) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int rr = m - 1 + k;
                            if (rr >= 0 && rr < n) v += wr[k] * colcol[split_idx<KR>(kColPad + rr, HC)];
                        }
                        if (clamp) {
                            const float a0 = m >= 0 ? colcol[split_idx<KR>(kColPad + m, HC)] : 0.f;
                            const float a1 = m + 1 < n ? colcol[split_idx<KR>(kColPad + m + 1, HC)] : 0.f;
                            v = clamp_to(v, fminf(a0, a1), fmaxf(a0, a1));
                        }
                    }
                    colbcol[split_idx<KR>(kColPad + y, HC)] = v;
                }
            }
            kcol = colbcol;
        }
        if (rot) {
            if constexpr (RS == 2) __syncthreads();  // both halves of every RF-kicked column
            else __syncwarp();
        }
        bool kick_ok = true;
        float4 kw = make_float4(0.f, 0.f, 0.f, 0.f);
        int s = 0;
        float csf = 1.f;  // the pending scale in the weights (clamp bounds)
        if (active && recs) {
            // the kick of column x and the pending scale of this step: the
            // finaliser CTA's records (lane 0 and lane 1 wait)
            unsigned r = 0;
            bool ok = true;
            if (lane < 2) ok = wait_tagged<1>(D, lane == 0 ? D.rword + x : D.sword + blockIdx.x, (unsigned)ps->k, &r);
            const unsigned rk = __shfl_sync(0xffffffffu, r, 0), rs = __shfl_sync(0xffffffffu, r, 1);
            kick_ok = __shfl_sync(0xffffffffu, (int)ok, 0) && __shfl_sync(0xffffffffu, (int)ok, 1);
            if (kick_ok) {
                const KickEntry e = kick_entry(__uint_as_float(rk), __uint_as_float(rs), ni);
                kw = e.w;
                s = e.s;
                csf = __uint_as_float(rs);
            } else if (lane == 0) {
                s_last = 1;
            }
        } else if (active) {
            const float4* kj = kbuf + 2 * W * (j & 3);
            kw = kj[0];
            s = __float_as_int(kj[1].x);
            csf = kj[1].y;
        }
        float lsum = 0.f;
        if (active && kick_ok) {
            float* dst = out + (size_t)x * ld;
            if (s >= -4 && s <= 4) {
                const int A2 = s - 2 + kColPad;  // column index of row y0+s-2, minus y0
                // A2 = s + 14 with |s| <= 4: (A2 & 7) = 5 and 6 are s = -1 and 0 only
                auto kick_rows = [&](int r0, int r1) -> float {
                    switch (KR == 8 ? (A2 & 7) : (A2 & 3)) {
                    case 0: return kick_fp_column<0, 0, KR, false, true, NI>(kcol, HC, gtab, dst, n, s, A2, kw, lane, clamp, csf, r0, r1);
                    case 1: return kick_fp_column<1, 0, KR, false, true, NI>(kcol, HC, gtab, dst, n, s, A2, kw, lane, clamp, csf, r0, r1);
                    case 2: return kick_fp_column<2, 0, KR, false, true, NI>(kcol, HC, gtab, dst, n, s, A2, kw, lane, clamp, csf, r0, r1);
                    case 3: return kick_fp_column<3, 0, KR, false, true, NI>(kcol, HC, gtab, dst, n, s, A2, kw, lane, clamp, csf, r0, r1);
                    case 4: return kick_fp_column<0, 1, KR, false, true, NI>(kcol, HC, gtab, dst, n, s, A2, kw, lane, clamp, csf, r0, r1);
                    case 5: return kick_fp_column<1, 1, KR, KR == 8, true, NI>(kcol, HC, gtab, dst, n, s, A2, kw, lane, clamp, csf, r0, r1);
                    case 6: return kick_fp_column<2, 1, KR, KR == 8, true, NI>(kcol, HC, gtab, dst, n, s, A2, kw, lane, clamp, csf, r0, r1);
                    default: return kick_fp_column<3, 1, KR, false, true, NI>(kcol, HC, gtab, dst, n, s, A2, kw, lane, clamp, csf, r0, r1);
                    }
                };
                if (RS == 1 && Y2 < n) lsum = kick_rows(0, Y2) + kick_rows(Y2, n);  // lower + upper half
                else lsum = kick_rows(ylo, yhi);
            } else {
                // large kick: plain per-row evaluation with bounds
                const float w[4] = {kw.x, kw.y, kw.z, kw.w};
                auto large_rows = [&](int r0, int r1) -> float {
                    float acc = 0.f;
                    for (int y = r0 + lane; y < r1; y += 32) {
                        float b[4];
#pragma unroll
                        for (int d = 0; d < 4; ++d) {
                            const int yy = y - 1 + d;
                            const int mm = yy + s;
                            float v = 0.f;
                            if (yy >= 0 && yy < n && mm > -2 && mm < n) {
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    const int rr = mm - 1 + k;
                                    if (rr >= 0 && rr < n) v = fmaf(w[k], kcol[split_idx<KR>(kColPad + rr, HC)], v);
                                }
                                if (clamp) {
                                    const float a0 = mm >= 0 ? kcol[split_idx<KR>(kColPad + mm, HC)] : 0.f;
                                    const float a1 = mm + 1 < n ? kcol[split_idx<KR>(kColPad + mm + 1, HC)] : 0.f;
                                    v = clamp_to(v, csf * fminf(a0, a1), csf * fmaxf(a0, a1));
                                }
                            }
                            b[d] = v;
                        }
                        const int gi = split_idx<KR>(y, n >> 3);
                        const float v = fp_apply(gtab[gi], gtab[n + gi], gtab[2 * n + gi], gtab[3 * n + gi], b);
                        dst[y] = v;
                        acc += v;
                    }
                    return acc;
                };
                if (RS == 1 && Y2 < n) lsum = large_rows(0, Y2) + large_rows(Y2, n);
                else lsum = large_rows(ylo, yhi);
            }
        }
        if constexpr (RS == 2) {
            // the column's lane partials: lower half (this warp, half 0) plus
            // upper half (its partner warp), in that order
            if (active && kick_ok && half == 1) xsum[32 * cw + lane] = lsum;
            __syncthreads();
            if (half == 0) lsum = lsum + xsum[32 * cw + lane];
        }
        if (active && kick_ok && half == 0) {
            // the column sum: FP32 lane partials, then an FP32 shuffle tree
            // (the state's precision, Sec. IV.A; an FP64 tree is five long
            // FP64 latencies on the path of every step on this GPU)
            float csum = lsum;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) csum += __shfl_down_sync(0xffffffffu, csum, o);
            if (lane == 0) {
                if constexpr (PERSIST) {
                    // the tagged word the finaliser CTA polls
                    st_tagged(D.cword + x, __float_as_uint(csum), (unsigned)ps->k + 1u);
                } else {
                    colsum[x] = double(csum);
                }
            }
        }
        __syncthreads();  // the ring slots of columns xs+jW-h .. xs+jW+W-h-1 are free
        if (PERSIST && s_last) {  // a kick record never came
            cp_async_wait_0();
            return false;
        }
        if (j + 2 < T) {
            load_columns<NW>(ring, R, P, RP, in, ld, n, xs + (j + 2) * W + h, W);
            if (!recs && half == 0) load_kick(kbuf + 2 * W * ((j + 2) & 3), kickw, xs + (j + 2) * W + cw, n, lane);
        }
        cp_async_commit();
    }
    cp_async_wait_0();
    // moment-recording steps: the p-moments of the strip's columns, read back
    // after the loop (every tile ended with a barrier, so all are written),
    // keeping the hot loop free of the extra work
    if (mom_now) strip_p_moments(D, out, xs, T * W, n, ld);
    // this thread's columns and column sums, before the ticket (persistent:
    // before the arrival count)
    if constexpr (PERSIST) fence_acq_rel_gpu();
    else __threadfence();
    __syncthreads();
    if constexpr (PERSIST) {
        // this CTA has written its columns of step k (its flag: k + 1)
        if (threadIdx.x == 0) asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(D.cflag + blockIdx.x),
                                           "r"((unsigned)ps->k + 1u) : "memory");
        return true;
    }
#ifdef VFPS_DEBUG
    if (threadIdx.x == 0 && s_dbg_site) D.st->status = -100 - s_dbg_site;
#endif
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(&D.st->ticket, 1u);
        s_last = (prev == (unsigned)(D.ntiles - 1));
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        finalise<float>(D, smem, 1);
    }
    return true;
}

// Streaming FP32 step.  CTA b walks its segments segs[b*spc .. b*spc+spc-1]
// in order, each (simulation, first column, tiles) a strip of strip_f32; a
// segment with no tiles ends the list.  With one segment per CTA the grid is
// one CTA per strip; with balanced segments every CTA takes an equal share of
// the launch's tiles, split at simulation boundaries.
// Resident CTAs per SM the register allocation is sized for (x W warps):
// 32 warps by default, i.e. 64 registers per thread.
#ifndef VFPS_FAST_WARPS_PER_SM
#define VFPS_FAST_WARPS_PER_SM 32
#endif

// Threads of a CTA of the FP32 step kernel: W warps, two per column for the
// N = 512 and 1024 instances (RS = 2 in strip_f32; the persistent kernel
// too).
__host__ __device__ constexpr int fast_threads(int W, int NC) { return W * 32 * (NC >= 512 ? 2 : 1); }

template <int W, int KR, int NC, int ROT, int NI = 4>
__global__ void __launch_bounds__(fast_threads(W, NC), VFPS_FAST_WARPS_PER_SM * 32 / fast_threads(W, NC))
step_kernel_f32(const Desc<float>* __restrict__ descs, const int4* __restrict__ segs, int spc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_last;
#ifdef VFPS_DEBUG
    if (threadIdx.x == 0) s_dbg_site = 0;
    __syncthreads();
#endif
    pdl_trigger();
    for (int i = 0; i < spc; ++i) {
        const int4 sg = segs[blockIdx.x * spc + i];
        if (sg.z <= 0) break;
        if (i > 0) __syncthreads();  // shared memory of the previous strip (or its finaliser) is free
        strip_f32<W, KR, NC, ROT, false, NI>(descs[sg.x], sg.y, sg.z, smem, s_last);
    }
}

// Persistent step of one lone simulation: K steps in one cooperative launch
// (all CTAs resident).  CTAs 0 .. G-2 are workers, one strip each of T tiles
// (segs, as for step_kernel_f32 with one segment per CTA, all of one length);
// CTA G-1 is the finaliser.  Before the launch the host sets every worker's
// step flag and every tagged word (column sums, kick records) to 0.
//  * Worker b, step k: wait until the workers whose columns its window reads
//    (columns xs - h .. xs + W T + h - 1) have finished step k-1 (flags >=
//    k: those columns of psi_k are written, and those CTAs no longer read
//    the columns this step overwrites -- the windows are symmetric); load
//    and rotate; for k > 0 wait for the column's kick record and the CTA's
//    scale word tagged k; kick, damp and diffuse; write the column sums
//    (two words each, tagged k+1); fence; flag k+1.
//  * Finaliser, step k: take each column sum as soon as both its words carry
//    tag k+1; on moment-recording steps also wait for every worker's flag (the
//    p-moment sums); run the finaliser arithmetic of the ticketed kernel
//    (finalise_compute: charge, scale, transforms, wake, power, series, step
//    count, parity), which also writes the kick records tagged k+1.
// The tagged words need no fence: only the step flags, which publish psi,
// are released with one (off the critical path while a worker rotates).
// So the transform of step k runs while the workers load and rotate step
// k+1, with the same arithmetic in the same order as K launches of
// step_kernel_f32; the twiddles and impedance stay in shared memory for the
// whole launch.  Every wait is bounded (spin_limit polls) and gives up with
// status VFPS_ETIMEOUT; the other CTAs then give up within 64 polls.
template <int W, int KR, int NC, int ROT>
__global__ void __launch_bounds__(fast_threads(W, NC), 1)
step_persistent_f32(const Desc<float>* __restrict__ descs, const int4* __restrict__ segs, int K)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_flag, s_fail;
    // the descriptor, in shared memory for the whole launch: the waits' fences
    // and asm memory clobbers would otherwise make every later field read a
    // fresh global load, after an acquire an L2 round trip
    __shared__ __align__(16) Desc<float> sD;
    {
        const int* src = reinterpret_cast<const int*>(descs);
        int* dst = reinterpret_cast<int*>(&sD);
        for (int i = threadIdx.x; i < (int)(sizeof(Desc<float>) / 4); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
    }
    const Desc<float>& D = sD;
    const int nwork = gridDim.x - 1;
    // parity and step count when the launch starts (the finaliser changes
    // both only after every worker has written its step-0 columns)
    const int par0 = D.st->parity;
    const long long t0 = D.st->t;
    if (blockIdx.x == gridDim.x - 1) {
        const int n = D.n;
        const FinSmem<float> L(smem, n, D.M / 2);
        finalise_load<float>(D, smem, true, false);
        for (int k = 0; k < K; ++k) {
            if (threadIdx.x == 0) s_fail = 0;
            __syncthreads();
            // the column sums as they arrive, and the transform input from them
            // (FP32 z_j = cs_2j + i cs_2j+1, zero-padded to M/2 values)
            float* z = reinterpret_cast<float*>(L.bufB);
            for (int x = threadIdx.x; x < D.M; x += blockDim.x) {
                if (x >= n) {
                    z[x] = 0.f;
                    continue;
                }
                unsigned v;
                if (!wait_tagged<1>(D, D.cword + x, (unsigned)k + 1u, &v)) {
                    s_fail = 1;
                    break;
                }
                const float c = __uint_as_float(v);
                L.cs[x] = double(c);
                z[x] = c;
            }
            __syncthreads();
            if (s_fail) return;
            const bool mom_now = D.mom_every > 0 && D.mring && (t0 + k + 1) % D.mom_every == 0;
            if (mom_now && !cta_wait_flags(D, 0, nwork - 1, (unsigned)k + 1u, &s_flag)) return;
            finalise_compute<float>(D, smem, 1, D.fault_no_signal ? 0u : (unsigned)(k + 1), nwork, true, k == K - 1);
        }
        return;
    }
    const int4 sg = segs[blockIdx.x];
    // workers whose columns this strip's window reads (strips of W sg.z columns)
    const int span = W * sg.z, h = D.h;
    const int c0 = max(0, (sg.y - h) / span), c1 = min(nwork - 1, (sg.y + span + h - 1) / span);
    PersistStep ps;
    for (int k = 0; k < K; ++k) {
        if (k > 0 && !cta_wait_flags(D, c0, c1, (unsigned)k, &s_flag)) return;
        ps.k = k;
        ps.par = par0 ^ (k & 1);
        ps.t = t0 + k;
        if (!strip_f32<W, KR, NC, ROT, true>(D, sg.y, sg.z, smem, s_fail, &ps)) return;
    }
}

}  // namespace vfps
