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
//   pring    ring of CSR powers, pring[t] = P(psi_t)
//   qring    ring of charges before renormalisation, qring[t] = Q of step t
//   st       DevState: pending scale, step count, ticket, parity, status
//
// The stored psi is the un-normalised result psi_c of the last step; the
// renormalisation factor Q0/Q is kept as the pending scale and applied when
// the next step stages psi into shared memory (Sec. "renormalisation").
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace vfps {

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
    int pad;
};

template <typename T>
struct Desc {
    T* psi[2];
    const typename C2<T>::type* zhat;
    const typename C2<T>::type* tw;
    double* colsum;
    double* rho;
    T* kick;
    double* pring;
    double* qring;
    DevState* st;
    int n, ld, M, logM;
    int ring_mask, renorm, clamp, h;  // h: column halo of the staged slab
    int ntiles;                        // CTAs per step of this instance
    int pad0;
    T cm1, sn, c;                      // cos(phi)-1, sin(phi), grid centre (n-1)/2
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
// Block-wide FP64 sum in a fixed order (deterministic), result to all threads.
__device__ __forceinline__ double block_sum(double v, double* red)
{
    int tid = threadIdx.x;
    red[tid] = v;
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
        if (tid < s) red[tid] += red[tid + s];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
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

// ----------------------------------------------------------------------------
// Finaliser: from the column sums of the state just written, compute the
// charge, the pending scale, the profile rho, its zero-padded M-point
// transform, the CSR power, and the wake/kick of the next step.
//   forward:  decimation-in-frequency radix-2 FFT, natural -> bit-reversed;
//   multiply by Zhat (Hermitian extension, DC and Nyquist dropped) in the
//             bit-reversed order, using rho~_{M-k} = conj(rho~_k) for real rho;
//   inverse:  decimation-in-time radix-2, bit-reversed -> natural.
// is_step = 1 after a time step (ring slot t+1, t advances); 0 for the
// prologue that only (re)computes the wake of the current state.
template <typename T>
__device__ void finalise(const Desc<T>& D, unsigned char* smem, int is_step)
{
    using T2 = typename C2<T>::type;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int n = D.n, M = D.M, K = M / 2, logM = D.logM;
    T2* a = reinterpret_cast<T2*>(smem);
    T2* tw = a + M;
    double* red = reinterpret_cast<double*>(tw + K);

    // charge Q = Delta^2 sum psi_c; colsum was written by other CTAs
    double part = 0.0;
    for (int x = tid; x < n; x += nt) part += __ldcg(D.colsum + x);
    double Q = D.delta * D.delta * block_sum(part, red);
    bool bad = !(Q > 0.0) || !isfinite(Q);
    double s_new = (D.renorm && !bad) ? 1.0 / Q : 1.0;

    for (int x = tid; x < M; x += nt) {
        double r = 0.0;
        if (x < n) {
            r = s_new * D.delta * __ldcg(D.colsum + x);
            D.rho[x] = r;
        }
        a[x] = T2{T(r), T(0)};
    }
    for (int k = tid; k < K; k += nt) tw[k] = D.tw[k];
    __syncthreads();

    // forward DIF
    for (int s = K; s >= 1; s >>= 1) {
        int stride = K / s;  // M/(2s)
        for (int b = tid; b < K; b += nt) {
            int j = b & (s - 1);
            int i = ((b - j) << 1) + j;
            T2 u = a[i], v = a[i + s];
            a[i] = cadd(u, v);
            a[i + s] = cmul(csub(u, v), tw[j * stride]);
        }
        __syncthreads();
    }

    // power and wake spectrum (bit-reversed positions)
    const T d = T(D.delta);
    double pp = 0.0;
    for (int pos = tid; pos < M; pos += nt) {
        int k = (int)(__brev((unsigned)pos) >> (32 - logM));
        T2 X = a[pos];
        X.x *= d;
        X.y *= d;  // rho~_k = Delta * X_k
        T2 B = {T(0), T(0)};
        if (k >= 1 && k < K) {
            T2 z = D.zhat[k];
            B = cmul(z, X);
            pp += 2.0 * double(z.x) * (double(X.x) * double(X.x) + double(X.y) * double(X.y));
        } else if (k > K) {
            T2 z = D.zhat[M - k];
            B = cmulc(X, z);  // conj(Z_{M-k}) rho~_k
        }
        a[pos] = B;
    }
    double P = D.dkappa * block_sum(pp, red);  // block_sum syncs

    // inverse DIT with conjugate twiddles
    for (int s = 1; s < M; s <<= 1) {
        int stride = K / s;
        for (int b = tid; b < K; b += nt) {
            int j = b & (s - 1);
            int i = ((b - j) << 1) + j;
            T2 w = tw[j * stride];
            w.y = -w.y;
            T2 u = a[i], v = cmul(a[i + s], w);
            a[i] = cadd(u, v);
            a[i + s] = csub(u, v);
        }
        __syncthreads();
    }
    for (int x = tid; x < n; x += nt) {
        double V = D.dkappa * double(a[x].x);
        D.kick[x] = T(D.kick_per_v * V);
    }
    if (tid == 0) {
        DevState* st = D.st;
        long long t = st->t;
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

    // rotation -> psi_a
    const int x = x0 + warp;
    const bool active = x < n;
    if (active) {
        T* ca = colA + warp * n;
        for (int y = lane; y < n; y += 32)
            ca[y] = rotate_cell<T, NI>(slab, P, x0 - h, x, y, n, D.cm1, D.sn, D.c, D.clamp);
    }
    __syncthreads();

    // kick -> psi_b : psi_b(y) = psi_a(y_r), y_r = y - kick[x]
    if (active) {
        const T* ca = colA + warp * n;
        T* cb = colB + warp * n;
        T ks = -D.kick[x];
        T fk = dfloor(ks);
        int sI = int(fk);
        T w[NI];
        lagrange_w<T, NI>(ks - fk, w);
        constexpr int F = -((NI - 1) / 2);
        for (int y = lane; y < n; y += 32) {
            int m = y + sI;
            T v = T(0);
            if (m > -2 && m < n) {
#pragma unroll
                for (int k = 0; k < NI; ++k) {
                    int r = m + F + k;
                    if (r >= 0 && r < n) v += w[k] * ca[r];
                }
                if (D.clamp) {
                    T a0 = (m >= 0) ? ca[m] : T(0);
                    T a1 = (m + 1 < n) ? ca[m + 1] : T(0);
                    v = clamp2(v, a0, a1);
                }
            }
            cb[y] = v;
        }
    }
    __syncwarp();

    // Fokker-Planck -> psi_c, column sum
    double csum = 0.0;
    if (active) {
        const T* cb = colB + warp * n;
        T* dst = out + (size_t)x * ld;
        T lsum = T(0);
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
        }
        csum = double(lsum);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) csum += __shfl_down_sync(0xffffffffu, csum, o);
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
    const T* in = D.psi[D.st->parity];
    if (x < n) {
        double s = 0.0;
        for (int y = lane; y < n; y += 32) s += double(in[(size_t)x * ld + y]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
            D.colsum[x] = s;
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

}  // namespace vfps
