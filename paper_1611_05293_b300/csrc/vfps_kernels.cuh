// vfps_kernels.cuh -- sm_103a kernels of one VFP time step.
//
// One launch advances every instance listed in its tile table by one time
// step (Sec. III.B of the paper: rotation, kick, damping/diffusion), and the
// last CTA of each instance computes that instance's next profile, wake and
// CSR power (Sec. II.B Eq. wakepotential, Sec. IV.C) -- the "last CTA per
// instance" finaliser, ordered by an atomic ticket and with no spin-wait.
//
// Layout (per instance, all in HBM):
//   psi[2]   n x ld values of T, row x = q_x, column y = p_y (p contiguous);
//            ping-pong buffers, device-side parity flips every step
//   zhat     M/2+1 complex T, dimensionless impedance at kappa_k
//   tw       M/2 complex T, exp(-2 pi i k/M)
//   colsum   n doubles, sum_y psi_c[x][y] of the step just written (scratch)
//   rho      n doubles, profile of the current (renormalised) state
//   kick     n T, p-shift of column x in grid cells for the next step
//   kickw    2n float4 (FP32 instances): per column x, [2x] the cubic weights
//            of that shift times the pending scale, [2x+1].x the node shift
//            floor(-kick) as int bits, [2x+1].y the pending scale (the clamp
//            bounds of a clamped kick)
//   pring    ring of CSR powers, pring[t] = P(psi_t)
//   qring    ring of charges before renormalisation, qring[t] = Q of step t
//   mring    (optional) ring of bunch moments, mring[4t..4t+3] = <q>, sigma_q,
//            <p>, sigma_p of psi_t for the recorded steps t
//   colmom   (moment steps) per column x: sum_y p_y psi_c, sum_y p_y^2 psi_c
//   st       DevState: pending scale, step count, ticket, parity, status
//
// The stored psi is the un-normalised result psi_c of the last step; the
// renormalisation factor Q0/Q is kept as the pending scale and applied when
// the next step stages psi into shared memory (Sec. "renormalisation").
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vfps {

// Index checks of the debug build (-DVFPS_DEBUG; the release build compiles
// them away): VFPS_GUARD(cond, site) is true when cond holds; otherwise it
// records the site in the CTA's s_dbg_site (first failure wins) and is false,
// and the caller skips the access.  The step kernel copies a recorded site to
// the instance's status word as -100 - site, which the host reports as
// VFPS_EBOUNDS.  A substitute for the memory checker, with no device fault.
#ifdef VFPS_DEBUG
__shared__ int s_dbg_site;
#define VFPS_GUARD(cond, site) ((cond) ? true : (atomicCAS(&::vfps::s_dbg_site, 0, (site)), false))
#else
#define VFPS_GUARD(cond, site) true
#endif

template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

struct DevState {
    double scale;        // pending renormalisation factor
    double qlast;        // charge before renormalisation of the last step
    long long t;         // steps done
    unsigned int ticket; // CTAs of the current step that have finished
    int parity;          // psi[parity] holds the current state
    int status;          // 0 or a negative VFPS_E* code
};

template <typename T>
struct Desc {
    T* psi[2];
    const typename C2<T>::type* zhat;
    const typename C2<T>::type* tw;
    double* colsum;                    // n column sums (scratch)
    double* rho;
    T* kick;
    float4* kickw;                     // FP32 path: 2 per column, see layout above
    double* pring;
    double* qring;
    double* mring;                     // moments ring (4 doubles per step), or null
    double* colmom;                    // 2n: per column sum p psi and sum p^2 psi (moment steps)
    // persistent launches (see step_persistent_f32): tagged words -- n
    // column sums (FP32), n kick records, a scale per worker CTA -- and a
    // step flag per worker CTA
    unsigned long long* cword;
    unsigned long long* rword;
    unsigned long long* sword;
    unsigned* cflag;
    DevState* st;
    int mom_every;                     // record moments of psi_t when t % mom_every == 0 (0: off)
    int ni;                            // interpolation points N_I (2, 3, 4)
    unsigned spin_limit;               // persistent launches: polls of a wait before VFPS_ETIMEOUT
    int fault_no_signal;               // test hook: the finaliser CTA never publishes (waits run out)
    int n, ld, M, logM;
    int ring_mask, renorm, clamp, h;  // h: column halo of the staged slab
    int ntiles;                        // CTAs per step of this instance
    int rotation;                      // 0 standard rotation, 1 Manhattan rotation
    T cm1, sn, c;                      // cos(phi)-1, sin(phi), grid centre (n-1)/2
    T hm;                              // Manhattan step h = 2 sin(pi/steps)
    T ga[4], gb[4];                    // FP increment weights g_k(y) = ga[k] + gb[k]*y
    double delta, dkappa;              // Delta, 2 pi/(M Delta)
    double kick_per_v;                 // S_csr * phi / Delta: grid cells per unit wake
};

// ----------------------------------------------------------------------------
// Lagrange weights on the nodes m+F .. m+F+NI-1, F = -floor((NI-1)/2),
// evaluated at the fraction t in [0, 1) (Eq. lagrange-basis-polynomials).
template <typename T, int NI>
__device__ __forceinline__ void lagrange_w(T t, T* w)
{
    if constexpr (NI == 4) {          // nodes -1, 0, 1, 2
        T tm1 = t - T(1), tm2 = t - T(2), tp1 = t + T(1);
        T a = t * tm1, b = tp1 * t;
        w[0] = -a * tm2 * T(1.0 / 6.0);
        w[1] = tp1 * tm1 * tm2 * T(0.5);
        w[2] = -b * tm2 * T(0.5);
        w[3] = b * tm1 * T(1.0 / 6.0);
    } else if constexpr (NI == 3) {   // nodes -1, 0, 1
        w[0] = t * (t - T(1)) * T(0.5);
        w[1] = (T(1) - t) * (T(1) + t);
        w[2] = t * (t + T(1)) * T(0.5);
    } else {                          // nodes 0, 1
        w[0] = T(1) - t;
        w[1] = t;
    }
}

// Lagrange weights of N_I = 2, 3 or 4 nodes (ni) in the 4-slot layout of the
// cubic stencil, nodes -1, 0, 1, 2 relative to floor: N_I = 3 takes nodes
// -1..1 and leaves slot 3 zero, N_I = 2 nodes 0..1 with slots 0 and 3 zero
// (the node sets of lagrange_w), so one window and one stencil serve every
// order (FP32 kernels).
__device__ __forceinline__ void lagrange_w4_rt(float t, float w[4], int ni)
{
    if (ni == 3) {
        float v[3];
        lagrange_w<float, 3>(t, v);
        w[0] = v[0];
        w[1] = v[1];
        w[2] = v[2];
        w[3] = 0.f;
    } else if (ni == 2) {
        float v[2];
        lagrange_w<float, 2>(t, v);
        w[0] = 0.f;
        w[1] = v[0];
        w[2] = v[1];
        w[3] = 0.f;
    } else {
        lagrange_w<float, 4>(t, w);
    }
}

template <typename T>
__device__ __forceinline__ T clamp2(T v, T a, T b)
{
    T lo = a < b ? a : b, hi = a < b ? b : a;
    return v < lo ? lo : (v > hi ? hi : v);
}

template <typename T> __device__ __forceinline__ T dfloor(T v);
template <> __device__ __forceinline__ float dfloor<float>(float v) { return floorf(v); }
template <> __device__ __forceinline__ double dfloor<double>(double v) { return floor(v); }

// ----------------------------------------------------------------------------
// Rotation of one cell (x, y) from the staged slab.  The source point is
// x_r = x + dx, y_r = y + dy with the displacement
//   dx = (cos phi - 1)(x - c) - sin phi (y - c),  dy = sin phi (x - c) + (cos phi - 1)(y - c),
// computed relative to the integer target so that FP32 keeps ~1e-7 cells.
// Sources more than one cell outside the grid give 0; off-grid nodes are 0.
template <typename T, int NI>
__device__ __forceinline__ T rotate_cell(const T* __restrict__ slab, int P, int cx0,
                                         int x, int y, int n, T cm1, T sn, T c, int clamp)
{
    T xc = T(x) - c, yc = T(y) - c;
    T dx = cm1 * xc - sn * yc;
    T dy = sn * xc + cm1 * yc;
    T fx = dfloor(dx), fy = dfloor(dy);
    int mx = x + int(fx), my = y + int(fy);
    if (mx <= -2 || mx >= n || my <= -2 || my >= n) return T(0);
    T wx[NI], wy[NI];
    lagrange_w<T, NI>(dx - fx, wx);
    lagrange_w<T, NI>(dy - fy, wy);
    constexpr int F = -((NI - 1) / 2);
    const T* base = slab + (mx + F - cx0) * P + (my + F + 2);
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < NI; ++a) {
        T r = T(0);
#pragma unroll
        for (int b = 0; b < NI; ++b) r += wy[b] * base[a * P + b];
        acc += wx[a] * r;
    }
    if (clamp) {
        const T* q = slab + (mx - cx0) * P + (my + 2);
        T v00 = q[0], v01 = q[1], v10 = q[P], v11 = q[P + 1];
        T lo = fmin(fmin(v00, v01), fmin(v10, v11));
        T hi = fmax(fmax(v00, v01), fmax(v10, v11));
        acc = acc < lo ? lo : (acc > hi ? hi : acc);
    }
    return acc;
}

// ----------------------------------------------------------------------------
// Manhattan rotation (Sec. III.B, symplectic rotation), first half: the drift
// q -> q + h p moves row y along q by h (y - c) cells, so the new value at
// (x, y) is the old one at x - h (y - c), interpolated along q from the
// staged slab.  As for the 2-D rotation, the displacement is formed first
// (small, exact in FP32 to ~1e-7 cells) and the node index from it.
template <typename T, int NI>
__device__ __forceinline__ T drift_cell(const T* __restrict__ slab, int P, int cx0, int x, int y, int n, T hm, T c,
                                        int clamp)
{
    const T dx = -hm * (T(y) - c);
    const T fx = dfloor(dx);
    const int mx = x + int(fx);
    if (mx <= -2 || mx >= n) return T(0);
    T w[NI];
    lagrange_w<T, NI>(dx - fx, w);
    constexpr int F = -((NI - 1) / 2);
    const T* base = slab + (mx + F - cx0) * P + (y + 2);
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < NI; ++a) acc += w[a] * base[a * P];
    if (clamp) acc = clamp2(acc, slab[(mx - cx0) * P + y + 2], slab[(mx + 1 - cx0) * P + y + 2]);
    return acc;
}

// One column shifted along p: dst(y) = src interpolated at y + shift (the RF
// kick of the Manhattan rotation, shift = h (x - c); the wake kick, shift =
// -kick).  Nodes off the grid are 0; a source more than one cell outside the
// grid gives 0; clamping restricts to the two nearest nodes.
template <typename T, int NI>
__device__ __forceinline__ void kick_column(const T* __restrict__ src, T* __restrict__ dst, T shift, int n, int clamp,
                                            int lane)
{
    const T fk = dfloor(shift);
    const int sI = int(fk);
    T w[NI];
    lagrange_w<T, NI>(shift - fk, w);
    constexpr int F = -((NI - 1) / 2);
    for (int y = lane; y < n; y += 32) {
        const int m = y + sI;
        T v = T(0);
        if (m > -2 && m < n) {
#pragma unroll
            for (int k = 0; k < NI; ++k) {
                const int r = m + F + k;
                if (r >= 0 && r < n) v += w[k] * src[r];
            }
            if (clamp) {
                const T a0 = (m >= 0) ? src[m] : T(0);
                const T a1 = (m + 1 < n) ? src[m + 1] : T(0);
                v = clamp2(v, a0, a1);
            }
        }
        dst[y] = v;
    }
}

// ----------------------------------------------------------------------------
// Programmatic dependent launch: a kernel lets the next kernel of its stream
// start as soon as all its CTAs are running (launch_dependents), and waits for
// the previous kernel to finish and flush (wait) only before touching what
// that kernel produced.  Without a programmatic dependency both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// 8- and 16-byte asynchronous global -> shared copies (cp.async).
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, int src_bytes)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Sum of v[0..count) in an order fixed by count alone (not by the block
// size, so a simulation gives the same bits whatever CTA width runs it): in
// blocks of 256 values, lane l takes v[l + 32 i], i = 0..7 (zeros past
// count) and adds them pairwise, ((0 + 1) + (2 + 3)) + ((4 + 5) + (6 + 7)),
// the blocks' lane values are added in order, then a shuffle tree.  Terms
// that are zero for every lane are left out (adding +0 changes no value), so
// a block takes 3 + 5 dependent adds at most, against up to 13 for a
// lane-sequential sum: FP64 adds have a long latency on this GPU.  Called by
// one whole warp; v is in shared memory and complete; lane 0 has the sum.
template <typename T>
__device__ __forceinline__ T warp_fixed_sum(const T* v, int count)
{
    const int lane = threadIdx.x & 31;
    T acc = T(0);
    for (int b = 0; b < count; b += 256) {
        const int rem = count - b;
        T a[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = (lane + 32 * i < rem) ? v[b + lane + 32 * i] : T(0);
        T t;
        if (rem > 128) t = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
        else if (rem > 64) t = (a[0] + a[1]) + (a[2] + a[3]);
        else if (rem > 32) t = a[0] + a[1];
        else t = a[0];
        acc = b ? acc + t : t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    return acc;
}

template <typename T2> __device__ __forceinline__ T2 cadd(T2 a, T2 b) { return {a.x + b.x, a.y + b.y}; }
template <typename T2> __device__ __forceinline__ T2 csub(T2 a, T2 b) { return {a.x - b.x, a.y - b.y}; }
template <typename T2> __device__ __forceinline__ T2 cmul(T2 a, T2 b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T2> __device__ __forceinline__ T2 cmulc(T2 a, T2 b)  // a * conj(b)
{
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

// Kick-table entry of a column whose p-shift for the next step is k cells,
// with the pending renormalisation factor sf folded into the weights:
// psi_b(y) = sum_j w_j psi_a(y + s - 1 + j) (N_I = ni nodes in the cubic
// layout, source y - k), s = floor(-k).  Both the finaliser and the persistent workers (which rebuild
// the entry from k and sf) compute it here.
struct KickEntry {
    float4 w;
    int s;
};
__device__ __forceinline__ KickEntry kick_entry(float k, float sf, int ni)
{
    const float ks = -k, fk = floorf(ks);
    float w[4];
    lagrange_w4_rt(ks - fk, w, ni);
    return {make_float4(sf * w[0], sf * w[1], sf * w[2], sf * w[3]), int(fk)};
}

// Tagged words of persistent launches: 64 bits, a 32-bit value in the low
// half and the launch step it belongs to (0: none yet) in the high half,
// stored and loaded as one (relaxed, GPU scope: single-copy atomic), so that
// a reader that sees the tag it waits for also sees that step's value -- no
// fence and no reset between steps.
__device__ __forceinline__ void st_tagged(unsigned long long* p, unsigned v, unsigned tag)
{
    const unsigned long long w = ((unsigned long long)tag << 32) | v;
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}
__device__ __forceinline__ unsigned long long ld_tagged(const unsigned long long* p)
{
    unsigned long long w;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(p) : "memory");
    return w;
}
// Acquire-release fence at GPU scope: with a relaxed store after it, a
// release; with a relaxed load before it, an acquire (lighter than
// __threadfence, which is sequentially consistent).
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// ----------------------------------------------------------------------------
// Finaliser: from the column sums of the state just written, compute the
// charge, the pending scale, the profile rho, its zero-padded M-point
// transform, the CSR power, and the wake/kick of the next step
// (Sec. II.B, Eq. wakepotential; Sec. IV.C for the power).
//
// rho is real, so one H = M/2 point complex transform does the work of the
// M-point one: z_j = rho_2j + i rho_2j+1 is transformed, split into the
// transforms of the even and odd samples (E_k = (Z_k + conj Z_{H-k})/2,
// O_k = (Z_k - conj Z_{H-k})/(2i)), and recombined, rho~_k = E_k + w^k O_k,
// w = exp(-2 pi i/M).  The wake spectrum B_k = Zhat_k rho~_k (k = 1..H-1;
// DC and Nyquist dropped, B_{M-k} = conj B_k) is folded back the same way,
// Y_k = (B_k + conj B_{H-k}) + i w^-k (B_k - conj B_{H-k}), so that the
// inverse H-point transform of Y gives V_2j + i V_2j+1.  Both transforms
// are Stockham radix-8 passes (a radix-4 or -2 pass last), natural order in
// and out, one barrier per pass.  Each output element is computed by the
// same operations whatever thread computes it, and the two sums use the
// fixed order of warp_fixed_sum, so the bits do not depend on the CTA width.
//
// is_step = 1 after a time step (ring slot t+1, t advances); 0 for the
// prologue that only (re)computes the wake of the current state.
// Shared memory (bytes) for FFT length M and n columns: two H-point complex
// buffers, twiddles (H) and impedance (H+1) complex values, the n column
// sums and H/2+1 power terms as doubles, and a reduction area.
// Groups of the finaliser's FP64 sums (sum_groups): for count values, the
// number of 256-value groups.
__host__ __device__ inline int sum_groups(int count) { return (count + 255) >> 8; }

__host__ __device__ inline size_t finalise_smem(int M, int n, int nt, int complex_bytes)
{
    (void)nt;
    const size_t H = (size_t)M / 2;
    const int G = sum_groups(n > (int)H / 2 + 1 ? n : (int)H / 2 + 1);
    return (4 * H + 2) * complex_bytes + (size_t)((n + 1) & ~1) * 8 + (H / 2 + 2) * 8 + (12 + 2 * (size_t)G) * 8;
}

template <typename T2, bool INV>
__device__ __forceinline__ T2 mul_mi(T2 a)  // a * (-i), or a * (+i) for the inverse
{
    return INV ? T2{-a.y, a.x} : T2{a.y, -a.x};
}

template <typename T2, bool INV>
__device__ __forceinline__ void dft4(T2& x0, T2& x1, T2& x2, T2& x3)
{
    const T2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = mul_mi<T2, INV>(csub(x1, x3));
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

// In-register R-point DFT (R = 2, 4, 8), exponent sign - (forward) or +.
template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_r(typename C2<T>::type* v)
{
    using T2 = typename C2<T>::type;
    if constexpr (R == 2) {
        const T2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        dft4<T2, INV>(v[0], v[1], v[2], v[3]);
    } else {
        dft4<T2, INV>(v[0], v[2], v[4], v[6]);  // E_0..E_3 of the even samples
        dft4<T2, INV>(v[1], v[3], v[5], v[7]);  // O_0..O_3 of the odd samples
        const T c = T(0.70710678118654752440);  // cos(pi/4)
        const T2 o1 = v[3], o3 = v[7];
        const T2 w1 = INV ? T2{c * (o1.x - o1.y), c * (o1.x + o1.y)} : T2{c * (o1.x + o1.y), c * (o1.y - o1.x)};
        const T2 w2 = mul_mi<T2, INV>(v[5]);
        const T2 w3 = INV ? T2{-c * (o3.x + o3.y), c * (o3.x - o3.y)} : T2{c * (o3.y - o3.x), -c * (o3.x + o3.y)};
        const T2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
        v[0] = cadd(e0, o0);
        v[4] = csub(e0, o0);
        v[1] = cadd(e1, w1);
        v[5] = csub(e1, w1);
        v[2] = cadd(e2, w2);
        v[6] = csub(e2, w2);
        v[3] = cadd(e3, w3);
        v[7] = csub(e3, w3);
    }
}

// One Stockham pass of an H-point transform: sub-transforms of length Ns =
// 2^lgNs are combined R at a time into length Ns*R.  tw[m] = exp(-2 pi i
// m/M), m < H.  Sizes are powers of two: shifts, not integer divisions (a
// division by a run-time value is a long dependent chain, and one transform
// runs in a single CTA, latency-bound).
template <typename T, int R, bool INV>
__device__ __forceinline__ void fft_pass(const typename C2<T>::type* __restrict__ src,
                                         typename C2<T>::type* __restrict__ dst,
                                         const typename C2<T>::type* __restrict__ tw, int H, int Ns, int lgNs,
                                         int t0 = threadIdx.x, int nthr = blockDim.x)
{
    using T2 = typename C2<T>::type;
    constexpr int lgR = R == 8 ? 3 : (R == 4 ? 2 : 1);
    const int Q = H >> lgR;
    const int mstep = (2 * H) >> (lgNs + lgR);  // twiddle r*k of this pass is exp(-2 pi i r k mstep/M)
    for (int j = t0; j < Q; j += nthr) {
        const int k = j & (Ns - 1);
        T2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[j + r * Q];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const int m = r * k * mstep;  // < 2H
                T2 w = tw[m < H ? m : m - H];
                if (m >= H) w = T2{-w.x, -w.y};
                if (INV) w.y = -w.y;
                v[r] = cmul(v[r], w);
            }
        }
        dft_r<T, R, INV>(v);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[base + r * Ns] = v[r];
    }
}

// H-point transform from src into one of the buffers x, y (out of place
// every pass); returns the buffer that holds the result.  after_first runs
// between the first pass and its barrier.
template <typename T, bool INV, typename F>
__device__ __forceinline__ typename C2<T>::type* fft_h(const typename C2<T>::type* src,
                                                       typename C2<T>::type* x, typename C2<T>::type* y,
                                                       const typename C2<T>::type* tw, int H, F after_first)
{
    using T2 = typename C2<T>::type;
    const T2* in = src;
    T2* out = x;
    T2* other = y;
    int Ns = 1, lgNs = 0;
    const int lgH = __ffs(H) - 1;
    bool first = true;
    while (Ns < H) {
        const int lgleft = lgH - lgNs;
        if (lgleft >= 3) {
            fft_pass<T, 8, INV>(in, out, tw, H, Ns, lgNs);
            lgNs += 3;
        } else if (lgleft == 2) {
            fft_pass<T, 4, INV>(in, out, tw, H, Ns, lgNs);
            lgNs += 2;
        } else {
            fft_pass<T, 2, INV>(in, out, tw, H, Ns, lgNs);
            lgNs += 1;
        }
        Ns = 1 << lgNs;
        if (first) after_first();
        first = false;
        __syncthreads();
        in = out;
        T2* t = out;
        out = other;
        other = t;
    }
    return const_cast<T2*>(in);
}

// The same transform on the first nthr threads of the block (whole warps),
// which synchronise among themselves on named barrier 1, so that the other
// warps can work meanwhile; every output is computed by the same operations
// as in fft_h.  Returns the buffer that holds the result (fft_result gives it
// to threads that did not take part).
__device__ __forceinline__ int fft_passes(int H)
{
    int p = 0;
    for (int lg = __ffs(H) - 1; lg > 0; lg -= (lg >= 3 ? 3 : lg)) ++p;
    return p;
}

template <typename T2>
__device__ __forceinline__ T2* fft_result(const T2* src, T2* x, T2* y, int H)
{
    const int p = fft_passes(H);
    return p == 0 ? const_cast<T2*>(src) : ((p & 1) ? x : y);
}

template <typename T, bool INV>
__device__ __forceinline__ typename C2<T>::type* fft_h_part(const typename C2<T>::type* src,
                                                            typename C2<T>::type* x, typename C2<T>::type* y,
                                                            const typename C2<T>::type* tw, int H, int nthr)
{
    using T2 = typename C2<T>::type;
    const T2* in = src;
    T2* out = x;
    T2* other = y;
    int lgNs = 0;
    const int lgH = __ffs(H) - 1, t0 = threadIdx.x;
    while (lgNs < lgH) {
        const int lgleft = lgH - lgNs, Ns = 1 << lgNs;
        if (lgleft >= 3) {
            fft_pass<T, 8, INV>(in, out, tw, H, Ns, lgNs, t0, nthr);
            lgNs += 3;
        } else if (lgleft == 2) {
            fft_pass<T, 4, INV>(in, out, tw, H, Ns, lgNs, t0, nthr);
            lgNs += 2;
        } else {
            fft_pass<T, 2, INV>(in, out, tw, H, Ns, lgNs, t0, nthr);
            lgNs += 1;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
        in = out;
        T2* t = out;
        out = other;
        other = t;
    }
    return const_cast<T2*>(in);
}

// Spectral step of the wake (Sec. II.B Eq. wakepotential), on the M/2-point
// transform Z of z_j = rho_2j + i rho_2j+1: for each pair of bins (k, H-k),
// H = M/2, split Z into the transforms of the even and odd samples, form the
// profile spectrum rho~_k = sk (E_k + w_k O_k) (w_k = exp(-2 pi i k/M)),
// multiply by the impedance, store the power term 2 Re Z_k |rho~_k|^2 (of k
// and H-k) in pterm[p] (if given), and fold the product back so that the
// inverse M/2-point transform gives the wake at the even and odd nodes.  DC
// and Nyquist carry no wake.  All threads of the block take part.
template <typename T>
__device__ __forceinline__ void wake_pair_pass(typename C2<T>::type* Z, const typename C2<T>::type* tw,
                                               const typename C2<T>::type* zh, int H, T sk, double* pterm, int tid,
                                               int nt)
{
    using T2 = typename C2<T>::type;
    for (int p = tid; p <= H / 2; p += nt) {
        T term = T(0);
        if (p == 0) {
            Z[0] = T2{T(0), T(0)};  // DC and Nyquist carry no wake
        } else {
            const int k = p, kk = H - p;
            const T2 zk = Z[k], zkk = Z[kk];
            const T2 E = {T(0.5) * (zk.x + zkk.x), T(0.5) * (zk.y - zkk.y)};
            const T2 O = {T(0.5) * (zk.y + zkk.y), T(0.5) * (zkk.x - zk.x)};
            const T2 w = tw[k];
            const T2 WO = cmul(w, O);
            const T2 rk = {sk * (E.x + WO.x), sk * (E.y + WO.y)};
            const T2 rkk = {sk * (E.x - WO.x), sk * (WO.y - E.y)};
            const T2 Zk = zh[k], Zkk = zh[kk];
            const T2 Bk = cmul(Zk, rk), Bkk = cmul(Zkk, rkk);
            term = T(2) * Zk.x * (rk.x * rk.x + rk.y * rk.y);
            if (kk != k) term += T(2) * Zkk.x * (rkk.x * rkk.x + rkk.y * rkk.y);
            const T2 S = {Bk.x + Bkk.x, Bk.y - Bkk.y};    // B_k + conj B_{H-k}
            const T2 Df = {Bk.x - Bkk.x, Bk.y + Bkk.y};   // B_k - conj B_{H-k}
            const T2 uD = cmulc(Df, w);                    // exp(+2 pi i k/M) * Df
            const T2 iuD = {-uD.y, uD.x};
            Z[k] = cadd(S, iuD);
            if (kk != k) Z[kk] = T2{S.x - iuD.x, iuD.y - S.y};  // conj(S - i u Df)
        }
        if (pterm) pterm[p] = double(term);
    }
}

// Moment sums of a recording step, on the finaliser's FP64 sum warp beside
// the forward transform: red[2..5] = sum q cs, sum q^2 cs (from the column
// sums cs in shared memory), sum of the per-column p psi and p^2 psi sums the
// step kernel wrote (colmom); each lane-sequential, then a shuffle tree.
__device__ __forceinline__ void moment_sums_warp(const double* cs, const double* colmom, int n, double delta,
                                                 double* red)
{
    const int lane = threadIdx.x & 31;
    const double cq = 0.5 * (n - 1);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    for (int x = lane; x < n; x += 32) {
        const double q = (x - cq) * delta, c = cs[x];
        a0 += q * c;
        a1 += q * q * c;
        a2 += __ldcg(colmom + 2 * x);
        a3 += __ldcg(colmom + 2 * x + 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_down_sync(0xffffffffu, a0, o);
        a1 += __shfl_down_sync(0xffffffffu, a1, o);
        a2 += __shfl_down_sync(0xffffffffu, a2, o);
        a3 += __shfl_down_sync(0xffffffffu, a3, o);
    }
    if (lane == 0) {
        red[2] = a0;
        red[3] = a1;
        red[4] = a2;
        red[5] = a3;
    }
}

// Shared-memory layout of the finaliser.
template <typename T>
struct FinSmem {
    using T2 = typename C2<T>::type;
    T2 *bufA, *bufB, *tw, *zh;
    double *cs, *pterm, *red;
    __device__ FinSmem(unsigned char* smem, int n, int H)
    {
        bufA = reinterpret_cast<T2*>(smem);
        bufB = bufA + H;
        tw = bufB + H;
        zh = tw + H;
        cs = reinterpret_cast<double*>(zh + H + 2);  // n column sums
        pterm = cs + ((n + 1) & ~1);                 // H/2+1 power terms
        red = pterm + H / 2 + 2;
    }
};

// One round of asynchronous copies into the finaliser's shared memory: the
// twiddles and impedance (tables), the column sums (written by the other
// CTAs of this step; .cg keeps L1 out of the way), or both.
template <typename T>
__device__ __forceinline__ void finalise_load(const Desc<T>& D, unsigned char* smem, bool tables, bool colsums)
{
    using T2 = typename C2<T>::type;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n = D.n, H = D.M / 2;
    const FinSmem<T> L(smem, n, H);
    constexpr int CB = sizeof(T2);
    const char* gtw = reinterpret_cast<const char*>(D.tw);
    const char* gzh = reinterpret_cast<const char*>(D.zhat);
    const char* gcs = reinterpret_cast<const char*>(D.colsum);
    const int ntw = H * CB / 16, zbytes = (H + 1) * CB, nzh = (zbytes + 15) / 16;
    const int cbytes = n * 8, ncs = (cbytes + 15) / 16;
    if (tables) {
        for (int i = tid; i < ntw; i += nt) cp_async16(reinterpret_cast<char*>(L.tw) + 16 * i, gtw + 16 * i, 16);
        for (int i = tid; i < nzh; i += nt)
            cp_async16(reinterpret_cast<char*>(L.zh) + 16 * i, gzh + 16 * i, min(16, zbytes - 16 * i));
    }
    if (colsums)
        for (int i = tid; i < ncs; i += nt)
            cp_async16(reinterpret_cast<char*>(L.cs) + 16 * i, gcs + 16 * i, min(16, cbytes - 16 * i));
    cp_async_commit();
    cp_async_wait_0();
    __syncthreads();
}

// The finaliser's arithmetic, from the column sums, twiddles and impedance
// in shared memory.  gen > 0 (persistent launches): also the kick records of
// the launch's step gen, tagged words D.rword[x] = (kick of column x, gen)
// and D.sword[b] = (pending scale, gen) for each worker CTA b < nscale,
// written before the rest of the table.  prepped: the caller has already
// written the transform input (zero-padded FP32 column sums) and synchronised.
// table = false leaves the kick table, the kicks and rho unwritten (a
// persistent launch's steps before its last, whose workers take the records).
template <typename T>
__device__ void finalise_compute(const Desc<T>& D, unsigned char* smem, int is_step, unsigned gen = 0,
                                 int nscale = 0, bool prepped = false, bool table = true)
{
    using T2 = typename C2<T>::type;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n = D.n, M = D.M, H = M / 2;
    const FinSmem<T> L(smem, n, H);
    T2* bufA = L.bufA;
    T2* bufB = L.bufB;
    T2* tw = L.tw;
    T2* zh = L.zh;
    double* cs = L.cs;
    double* pterm = L.pterm;
    double* red = L.red;

    // the step counter, read early (its latency overlaps the transforms)
    // (every thread reads it: the moment steps below depend on it, and thread
    // 0 only advances it after the last barrier)
    const long long t_now = D.st->t;
    // transform input z_j = cs_2j + i cs_2j+1 (zero-padded), in T
    if (!prepped) {
        for (int j = tid; j < H; j += nt) {
            const int x = 2 * j;
            bufB[j] = T2{x < n ? T(cs[x]) : T(0), x + 1 < n ? T(cs[x + 1]) : T(0)};
        }
        __syncthreads();
    }

    // Roles: the first warps (F) run the transforms, the wake pass and the
    // kick table; the last nsum warps (S) form the FP64 sums -- the charge,
    // then the power terms -- and the pending scale.  Each FP64 sum has a
    // structure fixed by its length alone: groups of 256 consecutive values,
    // each summed as warp_fixed_sum sums, then the group sums added in order;
    // the sum warps take the groups in turn, so the bits do not depend on how
    // many there are (nor on the CTA width).  FP64 arithmetic has a long
    // latency on this GPU, so in FP32 nothing of it lies on F's path: the
    // spectrum factor sk = 1/c (c = sum of the column sums, Delta^2 c = Q)
    // is the FP32 reciprocal of the forward transform's own DC bin, and F
    // waits for S only for the pending scale, after the inverse transform;
    // S's power sum ends beside the kick table.  (FP64: sk comes from the
    // FP64 scale, so F waits for it before the wake pass.)  A one-warp block
    // plays both roles in turn.  Named barriers: 1 among F, 2 among S, 3
    // (F arrives, S waits) wake pass done, 4 (S arrives, F waits) scale ready.
    constexpr bool f32 = sizeof(T) == 4;
    const int nw = nt >> 5, wid = tid >> 5;
    const int Gc = sum_groups(n), Gp = sum_groups(H / 2 + 1);
    const int nsum = nw == 1 ? 1 : max(1, min(max(Gc, Gp), nw / 2));
    const int sw = nw == 1 ? 0 : wid - (nw - nsum);  // index among the sum warps, < 0 for the others
    const bool solo = nw == 1;
    const bool sum_thread = sw >= 0, fft_thread = solo || sw < 0;
    const int nF = solo ? nt : nt - 32 * nsum, nFS = nt;
    double* gsum_c = red + 12;      // Gc group sums of the charge
    double* gsum_p = gsum_c + Gc;   // Gp group sums of the power terms
    float* skp = reinterpret_cast<float*>(red + 11);
    const bool mom_now = is_step && D.mom_every > 0 && D.mring && (t_now + 1) % D.mom_every == 0;
    T2* Z = fft_result<T2>(bufB, bufA, bufB, H);
    T2* const Zo = Z == bufA ? bufB : bufA;
    T2* y = fft_result<T2>(Z, Zo, Z, H);

    // S: the charge, the pending scale and profile factor (and, on a
    // recording step, the moment sums)
    auto charge_and_scale = [&]() {
        for (int g = sw; g < Gc; g += nsum) {
            const double sum = warp_fixed_sum<double>(cs + 256 * g, min(256, n - 256 * g));
            if ((tid & 31) == 0) gsum_c[g] = sum;
        }
        if (nsum > 1) asm volatile("bar.sync 2, %0;" ::"r"(32 * nsum) : "memory");
        if (tid == 32 * (nw - nsum)) {
            double c = gsum_c[0];
            for (int g = 1; g < Gc; ++g) c += gsum_c[g];
            const double q = D.delta * D.delta * c;
            const bool b = !(q > 0.0) || !isfinite(q);
            const double s1 = (D.renorm && !b) ? 1.0 / q : 1.0;
            red[0] = c;
            red[8] = q;
            red[9] = s1;
            red[10] = s1 * D.delta;
        }
        if (mom_now && sw == 0) moment_sums_warp(cs, D.colmom, n, D.delta, red);
    };
    // S: the power terms
    auto power_sum = [&]() {
        for (int g = sw; g < Gp; g += nsum) {
            const double sum = warp_fixed_sum<double>(pterm + 256 * g, min(256, H / 2 + 1 - 256 * g));
            if ((tid & 31) == 0) gsum_p[g] = sum;
        }
    };

    if (solo) {
        fft_h_part<T, false>(bufB, bufA, bufB, tw, H, nt);
        charge_and_scale();
        __syncwarp();
    } else if (sum_thread) {
        charge_and_scale();
        asm volatile("bar.arrive 4, %0;" ::"r"(nFS) : "memory");
        asm volatile("bar.sync 3, %0;" ::"r"(nFS) : "memory");
        power_sum();
    }
    if (fft_thread) {
        if (!solo) fft_h_part<T, false>(bufB, bufA, bufB, tw, H, nF);
        T sk;
        if constexpr (f32) {
            // 1/c from the DC bin (the sums of the even and odd column sums)
            if (tid == 0) {
                const float c = Z[0].x + Z[0].y;
                skp[0] = (D.renorm && c > 0.f && isfinite(c)) ? __frcp_rn(c) : float(D.delta * D.delta);
            }
            asm volatile("bar.sync 1, %0;" ::"r"(nF) : "memory");
            sk = skp[0];
        } else {
            if (!solo) asm volatile("bar.sync 4, %0;" ::"r"(nFS) : "memory");
            sk = T(red[10] * D.delta);  // rho~_k = Delta * DFT(rho)_k = sk * X_k
        }
        wake_pair_pass<T>(Z, tw, zh, H, sk, pterm, tid, nF);
        asm volatile("bar.sync 1, %0;" ::"r"(nF) : "memory");
        if (!solo) asm volatile("bar.arrive 3, %0;" ::"r"(nFS) : "memory");
        fft_h_part<T, true>(Z, Zo, Z, tw, H, nF);
        if (solo) power_sum();
        else if (f32) asm volatile("bar.sync 4, %0;" ::"r"(nFS) : "memory");

        // the kick table (and, in persistent launches, the tagged records
        // first) on F, from the inverse transform and the pending scale
        const double s_new = red[9];
        const double sd = red[10];  // rho_x = sd * cs_x
        const T kpv = T(D.kick_per_v * D.dkappa);
        if constexpr (f32) {
            if (gen) {
                for (int x = tid; x < n; x += nF) {
                    const T2 v = y[x >> 1];
                    st_tagged(D.rword + x, __float_as_uint(kpv * ((x & 1) ? v.y : v.x)), gen);
                }
                const unsigned sfb = __float_as_uint(float(s_new));
                for (int b = tid; b < nscale; b += nF) st_tagged(D.sword + b, sfb, gen);
            }
        }
        for (int x = tid; table && x < n; x += nF) {
            const T2 v = y[x >> 1];
            const T k = kpv * ((x & 1) ? v.y : v.x);
            D.kick[x] = k;
            D.rho[x] = sd * cs[x];
            if constexpr (f32) {
                const KickEntry e = kick_entry(k, float(s_new), D.ni);
                D.kickw[2 * x] = e.w;
                D.kickw[2 * x + 1] = make_float4(__int_as_float(e.s), float(s_new), 0.f, 0.f);
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        const double csum = red[0];
        const double Q = red[8];
        const bool bad = !(Q > 0.0) || !isfinite(Q);
        const double s_new = red[9];
        double psum = gsum_p[0];
        for (int g = 1; g < Gp; ++g) psum += gsum_p[g];
        const double P = D.dkappa * psum;
        DevState* st = D.st;
        const long long t = t_now;
        if (mom_now) {  // bunch length and energy spread of the new state (Sec. IV)
            const double s0 = csum, mq = red[2] / s0, mp = red[4] / s0;
            double* m = D.mring + 4 * ((t + 1) & D.ring_mask);
            m[0] = mq;
            m[1] = sqrt(fmax(red[3] / s0 - mq * mq, 0.0));
            m[2] = mp;
            m[3] = sqrt(fmax(red[5] / s0 - mp * mp, 0.0));
        }
        if (is_step) {
            D.qring[t & D.ring_mask] = Q;
            D.pring[(t + 1) & D.ring_mask] = P;
            st->t = t + 1;
            st->parity ^= 1;
            st->qlast = Q;
        } else {
            D.pring[t & D.ring_mask] = P;
        }
        st->scale = s_new;
        if (bad || !isfinite(P)) st->status = -5;
        st->ticket = 0u;
    }
}

template <typename T>
__device__ void finalise(const Desc<T>& D, unsigned char* smem, int is_step)
{
    finalise_load<T>(D, smem, true, true);
    finalise_compute<T>(D, smem, is_step, 0u);
}

// ----------------------------------------------------------------------------
// Fused step.  CTA = W columns x0..x0+W-1 of one instance, all rows; warp w
// owns column x0+w.  Shared memory: the slab of psi_t (scaled) for columns
// x0-h .. x0+W-1+h and rows -2 .. n+1 (zero outside the grid), then per warp
// one column of psi_a (rotation) and one of psi_b (kick, in the slab space
// once the rotation is done).  Epilogue: column sums of psi_c and the ticket.
template <typename T, int NI, int W>
__global__ void __launch_bounds__(W * 32)
step_kernel(const Desc<T>* __restrict__ descs, const int2* __restrict__ tiles)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_last;
    const int2 tile = tiles[blockIdx.x];
    const Desc<T>& D = descs[tile.x];
    const int x0 = tile.y;
    const int n = D.n, ld = D.ld, h = D.h;
    const int P = n + 4;                 // slab rows -2 .. n+1
    const int SW = W + 2 * h;            // slab columns
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    T* slab = reinterpret_cast<T*>(smem);
    T* colA = slab + SW * P;             // W columns of psi_a, n each
    T* colB = slab;                      // reuses the slab after the rotation

    pdl_trigger();
    pdl_wait();
    const int par = D.st->parity;
    const T scale = T(D.st->scale);
    const T* __restrict__ in = D.psi[par];
    T* __restrict__ out = D.psi[par ^ 1];

    // stage psi_t * scale
    for (int cx = warp; cx < SW; cx += W) {
        int gx = x0 - h + cx;
        bool colok = (gx >= 0 && gx < n);
        const T* src = in + (size_t)(colok ? gx : 0) * ld;
        for (int r = lane; r < P; r += 32) {
            int gy = r - 2;
            T v = T(0);
            if (colok && gy >= 0 && gy < n) v = scale * src[gy];
            slab[cx * P + r] = v;
        }
    }
    __syncthreads();

    // rotation -> psi_a (standard: 2-D; Manhattan: drift along q, then RF
    // kick along p), then the wake kick -> psi_b
    const int x = x0 + warp;
    const bool active = x < n;
    const T* cb;  // psi_b column of this warp
    if (D.rotation == 1) {
        if (active) {
            T* ca = colA + warp * n;
            for (int y = lane; y < n; y += 32)
                ca[y] = drift_cell<T, NI>(slab, P, x0 - h, x, y, n, D.hm, D.c, D.clamp);
        }
        __syncthreads();  // the slab is free: RF kick into it, wake kick back
        if (active) {
            kick_column<T, NI>(colA + warp * n, colB + warp * n, D.hm * (T(x) - D.c), n, D.clamp, lane);
            __syncwarp();
            kick_column<T, NI>(colB + warp * n, colA + warp * n, -D.kick[x], n, D.clamp, lane);
        }
        cb = colA + warp * n;
    } else {
        if (active) {
            T* ca = colA + warp * n;
            for (int y = lane; y < n; y += 32)
                ca[y] = rotate_cell<T, NI>(slab, P, x0 - h, x, y, n, D.cm1, D.sn, D.c, D.clamp);
        }
        __syncthreads();
        // kick -> psi_b : psi_b(y) = psi_a(y_r), y_r = y - kick[x]
        if (active) kick_column<T, NI>(colA + warp * n, colB + warp * n, -D.kick[x], n, D.clamp, lane);
        cb = colB + warp * n;
    }
    __syncwarp();

    // Fokker-Planck -> psi_c, column sum (and on moment-recording steps the
    // column's sums of p psi_c and p^2 psi_c, p_y = (y - c) Delta)
    const bool mom_now = D.mom_every > 0 && (D.st->t + 1) % D.mom_every == 0;
    double csum = 0.0;
    if (active) {
        T* dst = out + (size_t)x * ld;
        T lsum = T(0), lp1 = T(0), lp2 = T(0);
        const T dl = T(D.delta);
        const T ga0 = D.ga[0], ga1 = D.ga[1], ga2 = D.ga[2], ga3 = D.ga[3];
        const T gb0 = D.gb[0], gb1 = D.gb[1], gb2 = D.gb[2], gb3 = D.gb[3];
        for (int y = lane; y < n; y += 32) {
            T yf = T(y);
            T fm = (y >= 1) ? cb[y - 1] : T(0);
            T f0 = cb[y];
            T fp = (y + 1 < n) ? cb[y + 1] : T(0);
            T fpp = (y + 2 < n) ? cb[y + 2] : T(0);
            T inc = (ga0 + gb0 * yf) * fm + (ga1 + gb1 * yf) * f0 + (ga2 + gb2 * yf) * fp +
                    (ga3 + gb3 * yf) * fpp;
            T v = f0 + inc;
            dst[y] = v;
            lsum += v;
            if (mom_now) {
                const T pp = (yf - D.c) * dl, pv = pp * v;
                lp1 += pv;
                lp2 += pp * pv;
            }
        }
        {
            // lane partials, then a shuffle tree, in the state's precision
            T ct = lsum;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ct += __shfl_down_sync(0xffffffffu, ct, o);
            csum = double(ct);
        }
        if (mom_now) {
            double s1 = double(lp1), s2 = double(lp2);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                s1 += __shfl_down_sync(0xffffffffu, s1, o);
                s2 += __shfl_down_sync(0xffffffffu, s2, o);
            }
            if (lane == 0) {
                D.colmom[2 * x] = s1;
                D.colmom[2 * x + 1] = s2;
            }
        }
        if (lane == 0) {
            D.colsum[x] = csum;
            __threadfence();
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(&D.st->ticket, 1u);
        s_last = (prev == (unsigned)(D.ntiles - 1));
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        finalise<T>(D, smem, 1);
    }
}

// ----------------------------------------------------------------------------
// Prologue: column sums of the current state, then the finaliser (is_step=0).
// Used after create / set_state / set_impedance.  CTA = W columns.
template <typename T, int W>
__global__ void __launch_bounds__(W * 32)
project_kernel(const Desc<T>* __restrict__ descs, const int2* __restrict__ tiles)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_last;
    const int2 tile = tiles[blockIdx.x];
    const Desc<T>& D = descs[tile.x];
    const int n = D.n, ld = D.ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = tile.y + warp;
    pdl_trigger();
    pdl_wait();
    const T* in = D.psi[D.st->parity];
    if (x < n) {
        T ls = T(0);
        for (int y = lane; y < n; y += 32) ls += in[(size_t)x * ld + y];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ls += __shfl_down_sync(0xffffffffu, ls, o);
        if (lane == 0) {
            D.colsum[x] = double(ls);
            __threadfence();
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(&D.st->ticket, 1u);
        s_last = (prev == (unsigned)(D.ntiles - 1));
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        finalise<T>(D, smem, 0);
    }
}

// ----------------------------------------------------------------------------
// Bunch moments of the current state (the bunch length and energy spread of
// the paper's figures): <f> = sum f psi / sum psi over the nodes.
// Pass 1, one warp per column x: FP32 lane partials of psi, p psi, p^2 psi,
// summed across lanes in FP64 into m[3x .. 3x+2].  Pass 2, one CTA: fixed-
// order FP64 sums over the columns, out = {<q>, sigma_q, <p>, sigma_p}
// (m + 3n .. m + 3n + 3).  The stored psi carries a pending scale, which
// cancels in every ratio.
template <typename T, int W>
__global__ void __launch_bounds__(W * 32)
moments_columns_kernel(const Desc<T>* __restrict__ descs, const int2* __restrict__ tiles, double* __restrict__ m)
{
    const int2 tile = tiles[blockIdx.x];
    const Desc<T>& D = descs[tile.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = tile.y + warp, n = D.n;
    if (x >= n) return;
    const T* col = D.psi[D.st->parity] + (size_t)x * D.ld;
    const T L = T(D.c * D.delta), d = T(D.delta);  // p_y = -L + y Delta, L = c Delta
    T a0 = T(0), a1 = T(0), a2 = T(0);
    for (int y = lane; y < n; y += 32) {
        const T v = col[y], p = T(y) * d - L;
        const T pv = p * v;
        a0 += v;
        a1 += pv;
        a2 += p * pv;
    }
    double s0 = double(a0), s1 = double(a1), s2 = double(a2);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        m[3 * x] = s0;
        m[3 * x + 1] = s1;
        m[3 * x + 2] = s2;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) moments_finish_kernel(const Desc<T>* __restrict__ desc, double* __restrict__ m)
{
    const Desc<T>& D = *desc;
    const int n = D.n, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ double sums[5];
    if (warp < 5) {
        // warp 0: sum psi; 1: sum q psi; 2: sum q^2 psi; 3: sum p psi; 4: sum p^2 psi
        double acc = 0.0;
        for (int x = lane; x < n; x += 32) {
            const double q = (x - D.c) * D.delta;
            const double c0 = m[3 * x];
            acc += warp == 0 ? c0 : warp == 1 ? q * c0 : warp == 2 ? q * q * c0 : m[3 * x + warp - 2];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) sums[warp] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double mq = sums[1] / sums[0], mp = sums[3] / sums[0];
        double* out = m + 3 * n;
        out[0] = mq;
        out[1] = sqrt(fmax(sums[2] / sums[0] - mq * mq, 0.0));
        out[2] = mp;
        out[3] = sqrt(fmax(sums[4] / sums[0] - mp * mp, 0.0));
    }
}

// ----------------------------------------------------------------------------
// Power spectrum of L consecutive values of an instance's CSR-power series (a
// row of the paper's bursting spectrogram, Sec. IV.C): mean removed (FP64),
// Hann window, L-point complex FFT in FP32 (the Stockham passes of the
// finaliser), out[k] = |X_k|^2 for k = 0..L/2.  One CTA of 256 threads;
// shared memory 3 L float2 (two transform buffers and the twiddles
// exp(-pi i m/L), m < L).  P(psi_t) for t = t0 .. t0+L-1 sits in
// ring[t & mask].
__device__ __forceinline__ void window_spectrum(const double* __restrict__ ring, long long mask, long long t0, int L,
                                                double* __restrict__ out, unsigned char* smem, double* part)
{
    float2* A = reinterpret_cast<float2*>(smem);
    float2* B = A + L;
    float2* tw = B + L;
    const int tid = threadIdx.x;
    double acc = 0.0;
    for (int j = tid; j < L; j += 256) acc += ring[(t0 + j) & mask];
    part[tid] = acc;
    for (int m = tid; m < L; m += 256) {
        double sn, cs;
        sincospi(-(double)m / L, &sn, &cs);
        tw[m] = make_float2((float)cs, (float)sn);
    }
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (tid < h) part[tid] += part[tid + h];
        __syncthreads();
    }
    const double mean = part[0] / L;
    for (int j = tid; j < L; j += 256) {
        const double hann = 0.5 * (1.0 - cospi(2.0 * j / L));
        A[j] = make_float2((float)(hann * (ring[(t0 + j) & mask] - mean)), 0.f);
    }
    __syncthreads();
    float2* X = fft_h<float, false>(A, B, A, tw, L, [] {});
    for (int k = tid; k <= L / 2; k += 256) {
        const float2 v = X[k];
        out[k] = (double)v.x * v.x + (double)v.y * v.y;
    }
}

__global__ void __launch_bounds__(256)
power_spectrum_kernel(const double* __restrict__ ring, int mask, long long t0, int L, double* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double part[256];
    window_spectrum(ring, mask, t0, L, out, smem, part);
}

// One spectrogram window of one simulation per CTA: the series of simulation
// blockIdx.y starts its windows at t_first, window blockIdx.x at t_first +
// blockIdx.x hop; out[(y * count + x) * (L/2 + 1) ..].
struct SpecSeries {
    const double* ring;
    long long mask;
    long long t_first;
};

__global__ void __launch_bounds__(256)
spectrogram_kernel(const SpecSeries* __restrict__ series, int L, int hop, double* __restrict__ out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double part[256];
    const SpecSeries sr = series[blockIdx.y];
    const size_t row = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    window_spectrum(sr.ring, sr.mask, sr.t_first + (long long)blockIdx.x * hop, L, out + row * (L / 2 + 1), smem,
                    part);
}

// ----------------------------------------------------------------------------
// Host <-> device state transfers of many simulations at once.
//
// Upload: staged FP64 states (host copies in one block) are normalised to
// charge 1 on the device.  The charge of a state is summed in a fixed order
// that does not depend on how many states a call uploads: kStageParts
// consecutive parts of its n*n values, each summed by one CTA (thread t adds
// t, t+256, ... of its part, then a fixed tree), then the parts in order
// (stage_combine_kernel).  A part spread over kStageParts CTAs keeps a single
// upload short (FP64 adds are slow on this GPU).  Whether every value is
// finite is recorded beside: sums[2i] = charge sum, sums[2i+1] = 1 or 0.
constexpr int kStageParts = 16;

__global__ void __launch_bounds__(256)
stage_sum_kernel(const double* __restrict__ src, long long per_state, double* __restrict__ parts)
{
    __shared__ double part[256];
    __shared__ int bad;
    const long long lo = per_state * blockIdx.x / kStageParts, hi = per_state * (blockIdx.x + 1) / kStageParts;
    const double* v = src + (size_t)blockIdx.y * per_state;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    double acc = 0.0;
    bool fin = true;
    for (long long i = lo + threadIdx.x; i < hi; i += 256) {
        const double x = v[i];
        fin = fin && isfinite(x);
        acc += x;
    }
    part[threadIdx.x] = acc;
    if (!fin) bad = 1;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) part[threadIdx.x] += part[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* o = parts + 2 * ((size_t)blockIdx.y * kStageParts + blockIdx.x);
        o[0] = part[0];
        o[1] = bad ? 0.0 : 1.0;
    }
}

__global__ void __launch_bounds__(256)
stage_combine_kernel(const double* __restrict__ parts, int count, double* __restrict__ sums)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= count) return;
    const double* p = parts + 2 * (size_t)i * kStageParts;
    double acc = 0.0, ok = 1.0;
    for (int k = 0; k < kStageParts; ++k) {
        acc += p[2 * k];
        ok = p[2 * k + 1] == 1.0 ? ok : 0.0;
    }
    sums[2 * i] = acc;
    sums[2 * i + 1] = ok;
}

// One state of a transfer: its device psi (row pitch ld), grid size, and the
// factor applied on the way (upload: 1/(Delta^2 sum); download: read from st).
template <typename T>
struct StateJob {
    T* psi[2];
    DevState* st;        // parity; upload: the pending scale becomes 1, the ticket 0
    long long off;       // first value of this state in the staged block
    double delta2;       // upload: Delta^2
    int n, ld;
};

// Upload: psi[parity] = (T)(staged * inv), inv = 1/(Delta^2 sum), rows padded
// with zeros to ld; the state's pending scale becomes 1.  Grid (CTAs per
// state, states): CTA b takes rows b, b + gridDim.x, ...; the factor is
// formed once per CTA (an FP64 division is slow on this GPU).
template <typename T>
__global__ void __launch_bounds__(256)
stage_store_kernel(const double* __restrict__ src, const double* __restrict__ sums, const StateJob<T>* jobs)
{
    __shared__ double s_inv;
    const StateJob<T> j = jobs[blockIdx.y];
    if (threadIdx.x == 0) s_inv = 1.0 / (j.delta2 * sums[2 * blockIdx.y]);
    T* dst = j.psi[j.st->parity];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        j.st->scale = 1.0;
        j.st->ticket = 0u;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int x = blockIdx.x; x < j.n; x += gridDim.x) {
        const double* row = src + j.off + (long long)x * j.n;
        T* out = dst + (size_t)x * j.ld;
        for (int y = threadIdx.x; y < j.ld; y += blockDim.x) out[y] = y < j.n ? (T)(row[y] * inv) : T(0);
    }
}

// Download: staged[off + x n + y] = (double)psi[parity][x][y] * scale (the
// stored state with its pending renormalisation applied, as a single
// vfps_get_state computes it).  Grid (CTAs per state, states), rows as in
// stage_store_kernel.
template <typename T>
__global__ void __launch_bounds__(256)
stage_load_kernel(double* __restrict__ dst, const StateJob<T>* jobs)
{
    const StateJob<T> j = jobs[blockIdx.y];
    const T* src = j.psi[j.st->parity];
    const double scale = j.st->scale;
    for (int x = blockIdx.x; x < j.n; x += gridDim.x) {
        const T* row = src + (size_t)x * j.ld;
        double* out = dst + j.off + (long long)x * j.n;
        for (int y = threadIdx.x; y < j.n; y += blockDim.x) out[y] = (double)row[y] * scale;
    }
}

// Scatter of a staged block of small tables (twiddles, impedance, tile and
// segment lists, state word, descriptor) to their places in many
// instances' memory: one CTA per piece, 4-byte words (every piece is a
// multiple of 4 bytes and 4-byte aligned at both ends).
struct CopyJob {
    const unsigned int* src;
    unsigned int* dst;
    long long words;
};

__global__ void __launch_bounds__(128) scatter_kernel(const CopyJob* __restrict__ jobs)
{
    const CopyJob j = jobs[blockIdx.x];
    for (long long i = threadIdx.x; i < j.words; i += 128) j.dst[i] = j.src[i];
}

// Ring entries [lo_i, lo_i + cnt_i) of each state's CSR-power and charge
// rings into rows 2i and 2i+1 of a staged block (row r at out + r * cap),
// with the state's status word.
struct SeriesJob {
    const double* pring;
    const double* qring;
    const DevState* st;
    long long lo, cnt, mask;
};

__global__ void __launch_bounds__(256)
stage_series_kernel(double* __restrict__ out, long long cap, const SeriesJob* __restrict__ jobs,
                    int* __restrict__ status)
{
    const SeriesJob j = jobs[blockIdx.x];
    double* rp = out + (size_t)(2 * blockIdx.x) * cap;
    double* rq = rp + cap;
    for (long long i = threadIdx.x; i < j.cnt; i += 256) {
        rp[i] = j.pring[(j.lo + i) & j.mask];
        rq[i] = j.qring[(j.lo + i) & j.mask];
    }
    if (threadIdx.x == 0) status[blockIdx.x] = j.st->status;
}

}  // namespace vfps
