// vfps_pair.cuh -- FP32 step kernel that advances two simulations of the
// same geometry (grid, steps per period, damping) at once.
//
// The rotation map and the Fokker-Planck weights of such a pair are the same
// (Sec. III.A-B), so one lane computes a cell of both: the two states are
// interleaved element by element in shared memory, (psi_A, psi_B) of one
// node form a register pair, and every interpolation and stencil runs as
// packed FP32x2 arithmetic (sm_100+) with the shared weights broadcast into
// both halves.  Only the wake kick differs between the two (each has its own
// wake, Sec. II.A): its two 4-tap kernels are written as 5-tap kernels at the
// smaller of the two node shifts, with a zero at one end.
//
// Every value is computed with the same operations in the same order as
// step_kernel_f32 (vfps_fast.cuh) computes it for one simulation, so a
// simulation gives the same bits paired or alone (up to the sign of zeros).
//
// Shared-memory layouts (a "pair-row" is the 8 bytes (psi_A, psi_B) of one
// node; a "chunk" is 16 bytes, two pair-rows):
//  * ring slots: one slab column of both states, pair-rows -kPairRP ..
//    n+kPairRP-1, its chunks split into two sub-arrays (even chunks, odd
//    chunks): the lanes of a rotation pass read 4-row blocks, i.e. every
//    other chunk, and the split puts those reads on consecutive chunks;
//  * psi_a columns: kColPad zero pair-rows above and below, chunks split
//    four ways (chunk c at sub-array c & 3, index c >> 2) for the 8-row kick
//    blocks, sub-arrays 2 mod 4 chunks long so the rotation's stores spread
//    over all banks;
//  * FP weights: g_k(y) as broadcast pairs, chunk (row-in-block, tap pair)
//    major and block minor, so each lane reads its 8 rows conflict-free.
#pragma once
#include "vfps_fast.cuh"

namespace vfps {

// Asynchronous copy of one 4-byte element: the pair layout interleaves the
// two states element by element.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}

constexpr int kPairRP = 16;  // zero pair-rows above and below each ring column

// chunks per ring sub-array, bytes per ring slot (a multiple of 128 bytes:
// lanes that read different slots still meet distinct banks)
__host__ __device__ inline int pair_half(int n) { return (n + 2 * kPairRP) / 4; }
__host__ __device__ inline int pair_slot_bytes(int n) { return ((2 * pair_half(n) + 7) & ~7) * 16; }
// chunks per psi_a sub-array: covers n + 2 kColPad pair-rows, = 2 mod 4
__host__ __device__ inline int pair_cola_q(int n)
{
    const int q = (n + 2 * kColPad) / 8;
    return q + ((2 - q) & 3);
}

// Shared memory of the pair kernel: ring, psi_a columns, FP-weight table,
// 4-stage buffer of both simulations' kick-table entries.
__host__ inline size_t pair_ring_smem(int n, int h, int W)
{
    return (size_t)ring_slots(W, h) * pair_slot_bytes(n) + (size_t)W * 64 * pair_cola_q(n) + (size_t)32 * n +
           (size_t)256 * W;
}

// Slab columns col0 .. col0+ncols-1 of both states into their ring slots,
// element by element (rows 0..n-1; the padding pair-rows stay zero).  Lane l
// copies rows l, l+32, ...: pair-row l + kPairRP + 32 i sits in chunk
// (l >> 1) + 8 + 16 i, i.e. sub-array (l >> 1) & 1, index (l >> 2) + 4 + 8 i.
template <int W>
__device__ __forceinline__ void load_columns_pair(unsigned char* ring, int R, int SLOTB, int HALFB,
                                                  const float* __restrict__ inA, const float* __restrict__ inB,
                                                  int ld, int n, int col0, int ncols)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int off = ((lane >> 1) & 1) * HALFB + ((lane >> 2) + (kPairRP >> 2)) * 16 + (lane & 1) * 8;
    for (int k = warp; k < ncols; k += W) {
        const int gx = col0 + k;
        unsigned char* dst = ring + (gx & (R - 1)) * SLOTB + off;
        if (!VFPS_GUARD(off + (n / 32 - 1) * 128 + 8 <= SLOTB, 6)) continue;
        if (gx >= 0 && gx < n) {
            const float* a = inA + (size_t)gx * ld + lane;
            const float* b = inB + (size_t)gx * ld + lane;
            for (int i = 0; i < n / 32; ++i) {
                cp_async4(dst + 128 * i, a + 32 * i);
                cp_async4(dst + 128 * i + 4, b + 32 * i);
            }
        } else {
            for (int i = 0; i < n / 32; ++i) *reinterpret_cast<float2*>(dst + 128 * i) = f2(0.f, 0.f);
        }
    }
}

// Kick-table entries of column x of both simulations (lanes 0-1: A, 2-3: B).
__device__ __forceinline__ void load_kick_pair(float4* dst, const float4* __restrict__ kwA,
                                               const float4* __restrict__ kwB, int x, int n, int lane)
{
    if (lane < 4) {
        const float4* src = (lane < 2) ? kwA : kwB;
        const bool ok = x < n;
        cp_async16(dst + lane, ok ? src + 2 * x + (lane & 1) : src, ok ? 16 : 0);
    }
}

// Rotation of one cell of both states from the pair ring: the arithmetic of
// rotate_cell_ring in each half.
__device__ __forceinline__ float2 rotate_cell_pair(const unsigned char* __restrict__ ring, int R, int SLOTB,
                                                   int HALFB, int x, int y, int n, float cm1, float sn, float c)
{
    int mx, my;
    float wx[4], wy[4];
    if (!cell_weights<4>(x, y, n, cm1, sn, c, &mx, &my, wx, wy, 4)) return f2(0.f, 0.f);
    float2 acc = f2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const unsigned char* col = ring + ((mx - 1 + a) & (R - 1)) * SLOTB;
        float2 r = f2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int pr = my - 1 + b + kPairRP;
            const float2 v = *reinterpret_cast<const float2*>(col + ((pr >> 1) & 1) * HALFB + (pr >> 2) * 16 +
                                                              (pr & 1) * 8);
            r = __ffma2_rn(f2(wy[b], wy[b]), v, r);
        }
        acc = __ffma2_rn(f2(wx[a], wx[a]), r, acc);
    }
    return acc;
}

// Byte offset of pair-row pr of a psi_a column (four-way chunk split).
__device__ __forceinline__ int cola_pair_off(int pr, int QAB)
{
    const int cc = pr >> 1;
    return (cc & 3) * QAB + (cc >> 2) * 16 + (pr & 1) * 8;
}

// Rotation of column x of both states (rows 0..n-1, four per lane and pass)
// when the y-node offset FY is uniform (window alignment KA = K & 3, K = FY -
// 1 + kPairRP) and the x-node steps back by at most one inside a block of
// four rows: the arithmetic of rotate_column / rotate_block in each half.
// The 5-column window feeds two accumulations per row, over columns 1..4 (no
// step back) and 0..3 (stepped back), and the row keeps the one it needs.
template <int KA>
__device__ __forceinline__ void rotate_column_pair(const unsigned char* __restrict__ ring, int R, int SLOTB, int HALFB,
                                                   int K, unsigned char* __restrict__ colA, int QAB, int x, int n,
                                                   int lane, float xc, float c, float sn, float cm1, int FY)
{
    constexpr int O = KA & 1, Q = KA >> 1;
    const float2 msn2 = f2(-sn, -sn), cm12 = f2(cm1, cm1);
    const float2 snxc = f2(sn * xc, sn * xc), cmxc = f2(cm1 * xc, cm1 * xc);
    const float fyf = float(FY);
    const float2 mfy = f2(-fyf, -fyf);
    const int Kq = K >> 2;
    for (int yb = 0; yb < n; yb += 128) {
        const int y0 = yb + 4 * lane;
        if ((n & 127) && y0 >= n) break;
        const float yc0 = float(y0) - c;
        const float2 yc01 = f2(yc0, yc0 + 1.f), yc23 = f2(yc0 + 2.f, yc0 + 3.f);
        const float2 dx01 = __ffma2_rn(msn2, yc01, cmxc);
        const float2 dx23 = __ffma2_rn(msn2, yc23, cmxc);
        const float2 ty01 = __fadd2_rn(__ffma2_rn(cm12, yc01, snxc), mfy);
        const float2 ty23 = __fadd2_rn(__ffma2_rn(cm12, yc23, snxc), mfy);
        const float fx0 = floorf(dx01.x), fx1 = floorf(dx01.y), fx2 = floorf(dx23.x), fx3 = floorf(dx23.y);
        const float tx[4] = {dx01.x - fx0, dx01.y - fx1, dx23.x - fx2, dx23.y - fx3};
        const float ty[4] = {ty01.x, ty01.y, ty23.x, ty23.y};
        float2 wy[4][4], wx[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            lagrange2(f2(ty[k], ty[k]), wy[k]);
            lagrange2(f2(tx[k], tx[k]), wx[k]);
        }
        const int mx0 = x + int(fx0);
        const int slot0 = (mx0 - 2) & (R - 1);  // window columns mx0-2 .. mx0+2
        const int lb = ((y0 >> 2) + Kq) * 16;
        const bool ok = VFPS_GUARD(lb + ((Q + 3) >> 1) * 16 + 16 <= HALFB && K >= 0, 7);
        float2 accf[4], accb[4];
#pragma unroll
        for (int a = 0; a < 5; ++a) {
            const unsigned char* cb = ring + ((slot0 + a) & (R - 1)) * SLOTB + lb;
            float2 win[8];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float4 q = ok ? *reinterpret_cast<const float4*>(cb + ((Q + v) & 1) * HALFB + ((Q + v) >> 1) * 16)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
                win[2 * v] = f2(q.x, q.y);
                win[2 * v + 1] = f2(q.z, q.w);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float2 r = __fmul2_rn(wy[k][0], win[O + k]);
                r = __ffma2_rn(wy[k][1], win[O + k + 1], r);
                r = __ffma2_rn(wy[k][2], win[O + k + 2], r);
                r = __ffma2_rn(wy[k][3], win[O + k + 3], r);
                if (a >= 1) accf[k] = (a == 1) ? __fmul2_rn(wx[k][0], r) : __ffma2_rn(wx[k][a - 1], r, accf[k]);
                if (k >= 1 && a <= 3) accb[k] = (a == 0) ? __fmul2_rn(wx[k][0], r) : __ffma2_rn(wx[k][a], r, accb[k]);
            }
        }
        float2 out[4] = {accf[0], fx1 < fx0 ? accb[1] : accf[1], fx2 < fx0 ? accb[2] : accf[2],
                         fx3 < fx0 ? accb[3] : accf[3]};
        // sources more than one cell outside the grid give 0
        if (!((mx0 >= 0) && (mx0 <= n - 1) && (y0 + FY >= -1) && (y0 + 3 + FY <= n - 1))) {
            const float fxk[4] = {fx0, fx1, fx2, fx3};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int mx = x + int(fxk[k]), my = y0 + k + FY;
                if (mx <= -2 || mx >= n || my <= -2 || my >= n) out[k] = f2(0.f, 0.f);
            }
        }
        // pair-rows kColPad + y0 .. + 3: chunks cA, cA + 1
        const int cA = (kColPad >> 1) + (y0 >> 1);
        if (VFPS_GUARD(((cA + 1) >> 2) * 16 + 16 <= QAB, 8)) {
            *reinterpret_cast<float4*>(colA + (cA & 3) * QAB + (cA >> 2) * 16) =
                make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
            *reinterpret_cast<float4*>(colA + ((cA + 1) & 3) * QAB + ((cA + 1) >> 2) * 16) =
                make_float4(out[2].x, out[2].y, out[3].x, out[3].y);
        }
    }
}

// Kick + Fokker-Planck of the lane's 8-row blocks of one column of both
// states: kick_fp_column<...,8,...> in each half.  The 5-tap kernel w5 acts
// on psi_a rows y + s_min - 2 .. y + s_min + 2 for psi_b(y); E = 14 + s_min
// (pair-row offset of the window, EQ = (E >> 1) & 3, O2 = E & 1).  store: bit
// 0 writes psi_A, bit 1 psi_B.  SMALL: both shifts are -1 or 0.
template <int EQ, int O2, bool SMALL>
__device__ __forceinline__ float2 kick_fp_pair(const unsigned char* __restrict__ colA, int QAB,
                                               const unsigned char* __restrict__ gtab, float* __restrict__ dstA,
                                               float* __restrict__ dstB, int n, int E, const float2 w5[5], int loA,
                                               int hiA, int loB, int hiB, int store, int lane)
{
    constexpr int NB = 11;  // psi_b rows y0-1 .. y0+9
    const int nb8 = n >> 3;
    float2 lsum = f2(0.f, 0.f);
    for (int y0 = 8 * lane; y0 < n; y0 += 256) {
        const unsigned char* base = colA + ((y0 >> 3) + ((E >> 1) >> 2)) * 16;
        const bool ok = VFPS_GUARD((y0 >> 3) + ((E >> 1) >> 2) + ((EQ + 7) >> 2) < (QAB >> 4), 9);
        float2 win[16];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const float4 q = ok ? *reinterpret_cast<const float4*>(base + ((EQ + v) & 3) * QAB + ((EQ + v) >> 2) * 16)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            win[2 * v] = f2(q.x, q.y);
            win[2 * v + 1] = f2(q.z, q.w);
        }
        float2 b[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            float2 v = __fmul2_rn(w5[0], win[O2 + j]);
            v = __ffma2_rn(w5[1], win[O2 + j + 1], v);
            v = __ffma2_rn(w5[2], win[O2 + j + 2], v);
            v = __ffma2_rn(w5[3], win[O2 + j + 3], v);
            b[j] = __ffma2_rn(w5[4], win[O2 + j + 4], v);
        }
        if constexpr (SMALL) {
            if (y0 == 0) b[0] = f2(0.f, 0.f);
            if (y0 + 8 == n) {
                b[NB - 2] = f2(0.f, 0.f);
                b[NB - 1] = f2(0.f, 0.f);
            }
        } else {
            const int jloA = loA - y0 + 1, jhiA = hiA - y0 + 1, jloB = loB - y0 + 1, jhiB = hiB - y0 + 1;
#pragma unroll
            for (int j = 0; j < NB; ++j)
                b[j] = f2((j >= jloA && j <= jhiA) ? b[j].x : 0.f, (j >= jloB && j <= jhiB) ? b[j].y : 0.f);
        }
        float2 cc[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const float4 g01 = *reinterpret_cast<const float4*>(gtab + ((2 * r) * nb8 + (y0 >> 3)) * 16);
            const float4 g23 = *reinterpret_cast<const float4*>(gtab + ((2 * r + 1) * nb8 + (y0 >> 3)) * 16);
            float2 v = __fmul2_rn(f2(g01.x, g01.y), b[r]);
            v = __ffma2_rn(f2(g01.z, g01.w), b[r + 1], v);
            v = __ffma2_rn(f2(g23.x, g23.y), b[r + 2], v);
            cc[r] = __ffma2_rn(f2(g23.z, g23.w), b[r + 3], v);
        }
        if (store & 1) {
            *reinterpret_cast<float4*>(dstA + y0) = make_float4(cc[0].x, cc[1].x, cc[2].x, cc[3].x);
            *reinterpret_cast<float4*>(dstA + y0 + 4) = make_float4(cc[4].x, cc[5].x, cc[6].x, cc[7].x);
        }
        if (store & 2) {
            *reinterpret_cast<float4*>(dstB + y0) = make_float4(cc[0].y, cc[1].y, cc[2].y, cc[3].y);
            *reinterpret_cast<float4*>(dstB + y0 + 4) = make_float4(cc[4].y, cc[5].y, cc[6].y, cc[7].y);
        }
#pragma unroll
        for (int q4 = 0; q4 < 2; ++q4)
            lsum = __fadd2_rn(lsum, __fadd2_rn(__fadd2_rn(cc[4 * q4], cc[4 * q4 + 1]),
                                               __fadd2_rn(cc[4 * q4 + 2], cc[4 * q4 + 3])));
    }
    return lsum;
}

// Dispatch of kick_fp_pair on the window alignment.
__device__ __forceinline__ float2 kick_fp_pair_any(const unsigned char* colA, int QAB, const unsigned char* gtab,
                                                   float* dstA, float* dstB, int n, int E, const float2 w5[5],
                                                   int loA, int hiA, int loB, int hiB, int store, bool small,
                                                   int lane)
{
#define VFPS_KFP(EQ, O2, SM) \
    kick_fp_pair<EQ, O2, SM>(colA, QAB, gtab, dstA, dstB, n, E, w5, loA, hiA, loB, hiB, store, lane)
    const int sel = (((E >> 1) & 3) << 1) | (E & 1);
    if (small) {
        // E = 13 or 14 (s_min = -1 or 0): (EQ, O2) = (2, 1) or (3, 0)
        return sel == 5 ? VFPS_KFP(2, 1, true) : VFPS_KFP(3, 0, true);
    }
    switch (sel) {
    case 0: return VFPS_KFP(0, 0, false);
    case 1: return VFPS_KFP(0, 1, false);
    case 2: return VFPS_KFP(1, 0, false);
    case 3: return VFPS_KFP(1, 1, false);
    case 4: return VFPS_KFP(2, 0, false);
    case 5: return VFPS_KFP(2, 1, false);
    case 6: return VFPS_KFP(3, 0, false);
    default: return VFPS_KFP(3, 1, false);
    }
#undef VFPS_KFP
}

// Kick + FP of one state (half h of the pair) with a shift beyond 4 cells:
// the plain per-row evaluation of step_kernel_f32 on the pair layout.
__device__ __forceinline__ float kick_fp_large(const unsigned char* __restrict__ colA, int QAB,
                                               const unsigned char* __restrict__ gtab, float* __restrict__ dst,
                                               int n, int s, float4 kw, int h, int lane)
{
    const float w[4] = {kw.x, kw.y, kw.z, kw.w};
    const int nb8 = n >> 3;
    float lsum = 0.f;
    for (int y = lane; y < n; y += 32) {
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
                    if (rr >= 0 && rr < n)
                        v = fmaf(w[k], *reinterpret_cast<const float*>(colA + cola_pair_off(kColPad + rr, QAB) + 4 * h),
                                 v);
                }
            }
            b[d] = v;
        }
        float g[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            g[k] = *reinterpret_cast<const float*>(gtab + (((y & 7) * 2 + (k >> 1)) * nb8 + (y >> 3)) * 16 + (k & 1) * 8);
        const float v = fp_apply(g[0], g[1], g[2], g[3], b);
        dst[y] = v;
        lsum += v;
    }
    return lsum;
}

// One strip of the pair kernel: T consecutive W-column tiles of the pair
// (DA, DB) from column xs, walked as strip_f32 walks one simulation's strip;
// at the end the CTA takes a ticket of each simulation and runs the
// finaliser of each one it completes.
template <int W, int NC>
__device__ __forceinline__ void strip_f32x2(const Desc<float>& DA, const Desc<float>& DB, int xs, int T,
                                            unsigned char* smem, int* s_last)
{
    const int n = NC ? NC : DA.n, ld = NC ? NC : DA.ld, h = DA.h;
    const int R = ring_slots(W, h);
    const int SLOTB = pair_slot_bytes(n), HALFB = 16 * pair_half(n);
    const int QAB = 16 * pair_cola_q(n), CAB = 4 * QAB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float cm1 = DA.cm1, sn = DA.sn, c = DA.c;

    unsigned char* ring = smem;
    unsigned char* colA = ring + R * SLOTB + warp * CAB;  // this warp's psi_a column pair
    unsigned char* gtab = ring + R * SLOTB + W * CAB;
    float4* kbuf = reinterpret_cast<float4*>(gtab + 32 * n) + 4 * warp;  // stage k: kbuf + 4 W k

    // padding pair-rows of every ring slot (chunks 0..7 and n/2+8 .. n/2+15)
    // and of this warp's psi_a column: zero for the whole strip
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int slot = warp; slot < R; slot += W)
        if (lane < 16) {
            const int cc = lane < 8 ? lane : n / 2 + lane;
            *reinterpret_cast<float4*>(ring + slot * SLOTB + (cc & 1) * HALFB + (cc >> 1) * 16) = z4;
        }
    for (int cc = lane; cc < CAB / 16; cc += 32)
        if (cc < (kColPad >> 1) || cc >= (kColPad >> 1) + n / 2)
            *reinterpret_cast<float4*>(colA + (cc & 3) * QAB + (cc >> 2) * 16) = z4;
    for (int e = threadIdx.x; e < 4 * n; e += blockDim.x) {
        const int y = e >> 2, k = e & 3;
        const float g = fp_weight(DA, k, y);
        *reinterpret_cast<float2*>(gtab + (((y & 7) * 2 + (k >> 1)) * (n >> 3) + (y >> 3)) * 16 + (k & 1) * 8) =
            f2(g, g);
    }
    // what the previous steps wrote (state words, psi, kick tables) is read from here on
    pdl_wait();
    const int parA = DA.st->parity, parB = DB.st->parity;
    const float* __restrict__ inA = DA.psi[parA];
    const float* __restrict__ inB = DB.psi[parB];
    float* __restrict__ outA = DA.psi[parA ^ 1];
    float* __restrict__ outB = DB.psi[parB ^ 1];
    load_columns_pair<W>(ring, R, SLOTB, HALFB, inA, inB, ld, n, xs - h, W + 2 * h);
    load_kick_pair(kbuf, DA.kickw, DB.kickw, xs + warp, n, lane);
    cp_async_commit();
    if (T > 1) {
        load_columns_pair<W>(ring, R, SLOTB, HALFB, inA, inB, ld, n, xs + W + h, W);
        load_kick_pair(kbuf + 4 * W, DA.kickw, DB.kickw, xs + W + warp, n, lane);
    }
    cp_async_commit();

    for (int j = 0; j < T; ++j) {
        const int x = xs + j * W + warp;
        const bool active = x < n;
        cp_async_wait_1();
        __syncthreads();
        if (active) {
            const float xc = float(x) - c;
            const float fy_top = floorf(fmaf(cm1, 0.f - c, sn * xc));
            const float fy_bot = floorf(fmaf(cm1, float(n - 1) - c, sn * xc));
            if (fy_top == fy_bot && sn < 0.3f) {
                const int FY = int(fy_top);
                const int K = FY - 1 + kPairRP;
                switch (K & 3) {
                case 0: rotate_column_pair<0>(ring, R, SLOTB, HALFB, K, colA, QAB, x, n, lane, xc, c, sn, cm1, FY); break;
                case 1: rotate_column_pair<1>(ring, R, SLOTB, HALFB, K, colA, QAB, x, n, lane, xc, c, sn, cm1, FY); break;
                case 2: rotate_column_pair<2>(ring, R, SLOTB, HALFB, K, colA, QAB, x, n, lane, xc, c, sn, cm1, FY); break;
                default: rotate_column_pair<3>(ring, R, SLOTB, HALFB, K, colA, QAB, x, n, lane, xc, c, sn, cm1, FY); break;
                }
            } else {
                for (int y = lane; y < n; y += 32)
                    *reinterpret_cast<float2*>(colA + cola_pair_off(kColPad + y, QAB)) =
                        rotate_cell_pair(ring, R, SLOTB, HALFB, x, y, n, cm1, sn, c);
            }
        }
        __syncwarp();
        if (active) {
            const float4* kj = kbuf + 4 * W * (j & 3);
            const float4 kwA = kj[0], kwB = kj[2];
            const int sA = __float_as_int(kj[1].x), sB = __float_as_int(kj[3].x);
            float* dstA = outA + (size_t)x * ld;
            float* dstB = outB + (size_t)x * ld;
            const int loA = max(0, -1 - sA), hiA = min(n - 1, n - 1 - sA);
            const int loB = max(0, -1 - sB), hiB = min(n - 1, n - 1 - sB);
            float2 lsum;
            if (sA >= -4 && sA <= 4 && sB >= -4 && sB <= 4 && abs(sA - sB) <= 1) {
                // both kernels as 5-tap kernels at the smaller shift
                const int smin = min(sA, sB);
                const float wa[4] = {kwA.x, kwA.y, kwA.z, kwA.w}, wb[4] = {kwB.x, kwB.y, kwB.z, kwB.w};
                float2 w5[5];
#pragma unroll
                for (int t = 0; t < 5; ++t) {
                    const float a = (sA == smin) ? (t < 4 ? wa[t] : 0.f) : (t > 0 ? wa[t - 1] : 0.f);
                    const float b = (sB == smin) ? (t < 4 ? wb[t] : 0.f) : (t > 0 ? wb[t - 1] : 0.f);
                    w5[t] = f2(a, b);
                }
                const bool small = smin >= -1 && max(sA, sB) <= 0;
                lsum = kick_fp_pair_any(colA, QAB, gtab, dstA, dstB, n, 14 + smin, w5, loA, hiA, loB, hiB, 3, small,
                                        lane);
            } else {
                // shifts too far apart (or large): each state on its own
                float part[2];
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int s = hh ? sB : sA;
                    const float4 kw = hh ? kwB : kwA;
                    if (s >= -4 && s <= 4) {
                        const float2 w5[5] = {f2(kw.x, kw.x), f2(kw.y, kw.y), f2(kw.z, kw.z), f2(kw.w, kw.w),
                                              f2(0.f, 0.f)};
                        const int lo = max(0, -1 - s), hi = min(n - 1, n - 1 - s);
                        const float2 l2 = kick_fp_pair_any(colA, QAB, gtab, dstA, dstB, n, 14 + s, w5, lo, hi, lo, hi,
                                                           1 << hh, s >= -1 && s <= 0, lane);
                        part[hh] = hh ? l2.y : l2.x;
                    } else {
                        part[hh] = kick_fp_large(colA, QAB, gtab, hh ? dstB : dstA, n, s, kw, hh, lane);
                    }
                }
                lsum = f2(part[0], part[1]);
            }
            // FP32 lane partials and shuffle tree: lanes 0-15 reduce A, 16-31
            // B, in the order of the single-simulation tree (16, 8, 4, 2, 1)
            const bool upper = lane >= 16;
            float v = upper ? lsum.y : lsum.x;
            v += __shfl_xor_sync(0xffffffffu, upper ? lsum.x : lsum.y, 16);
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) DA.colsum[x] = double(v);
            if (lane == 16) DB.colsum[x] = double(v);
        }
        __syncthreads();  // the ring slots of columns xs+jW-h .. xs+jW+W-h-1 are free
        if (j + 2 < T) {
            load_columns_pair<W>(ring, R, SLOTB, HALFB, inA, inB, ld, n, xs + (j + 2) * W + h, W);
            load_kick_pair(kbuf + 4 * W * ((j + 2) & 3), DA.kickw, DB.kickw, xs + (j + 2) * W + warp, n, lane);
        }
        cp_async_commit();
    }
    cp_async_wait_0();
    __threadfence();  // this thread's column sums, before the tickets
    __syncthreads();
#ifdef VFPS_DEBUG
    if (threadIdx.x == 0 && s_dbg_site) {
        DA.st->status = -100 - s_dbg_site;
        DB.st->status = -100 - s_dbg_site;
    }
#endif
    if (threadIdx.x == 0) {
        s_last[0] = atomicAdd(&DA.st->ticket, 1u) == (unsigned)(DA.ntiles - 1);
        s_last[1] = atomicAdd(&DB.st->ticket, 1u) == (unsigned)(DB.ntiles - 1);
    }
    __syncthreads();
    if (s_last[0]) {
        __threadfence();
        finalise<float>(DA, smem, 1);
    }
    if (s_last[1]) {
        __syncthreads();
        __threadfence();
        finalise<float>(DB, smem, 1);
    }
}

// Streaming FP32 step of pairs of simulations: CTA b walks its segments
// segs[b*spc ..] (pair index, first column, tiles) as step_kernel_f32 walks
// its own; pair k is descriptors 2k and 2k+1.
template <int W, int NC>
__global__ void __launch_bounds__(W * 32, 16 / W)
step_kernel_f32x2(const Desc<float>* __restrict__ descs, const int4* __restrict__ segs, int spc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_last[2];
#ifdef VFPS_DEBUG
    if (threadIdx.x == 0) s_dbg_site = 0;
    __syncthreads();
#endif
    pdl_trigger();
    for (int i = 0; i < spc; ++i) {
        const int4 sg = segs[blockIdx.x * spc + i];
        if (sg.z <= 0) break;
        if (i > 0) __syncthreads();
        strip_f32x2<W, NC>(descs[2 * sg.x], descs[2 * sg.x + 1], sg.y, sg.z, smem, s_last);
    }
}

}  // namespace vfps
