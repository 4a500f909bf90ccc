// vfps_haissinski.cuh -- Haissinski equilibrium start on the device.
//
// Below the instability threshold the damped, diffused system relaxes to
// psi proportional to exp(-H) with H = (q^2 + p^2)/2 - S_csr Phi(q) and
// Phi' = V[rho], the wake potential of the profile itself (Sec. II.B Eq.
// wakepotential; Appendix A names the equilibrium).  The profile solves
//
//     rho(q) = A exp(-q^2/2 + S_csr int_{-L}^{q} V[rho](q') dq'),   Delta sum rho = 1,
//
// here by the damped fixed-point iteration rho <- (rho + new)/2 from the
// unit Gaussian, in FP64, one CTA per simulation: the wake is the step's own
// (same FFT length and impedance table, evaluated in FP64), the integral the
// trapezoid rule from q_0 = -L.  The state is then rho_H(q) g(p), g the unit
// Gaussian in p normalised on the grid.
#pragma once
#include "vfps_kernels.cuh"

namespace vfps {

// Shared memory of haissinski_kernel: two FFT buffers, twiddles and the
// impedance table as double2, three profiles of n doubles, scratch.
__host__ __device__ inline size_t haissinski_smem(int M, int n)
{
    const int H = M / 2;
    return (size_t)(4 * H + 1) * 16 + (size_t)3 * n * 8 + 64 * 8;
}

// Inclusive prefix sum of v[1..n-1] into out[i] = sum_{j=1..i} v[j], out[0] =
// 0, by one warp in a fixed order: lane l sums its contiguous chunk, the
// chunk totals are scanned across lanes, then each lane writes its chunk.
__device__ __forceinline__ void warp_prefix_trapezoid(const double* V, double* out, int n, double half_d)
{
    const int lane = threadIdx.x & 31;
    const int chunk = (n + 31) / 32;
    const int i0 = lane * chunk, i1 = min(n, i0 + chunk);
    double tot = 0.0;
    for (int i = max(i0, 1); i < i1; ++i) tot += half_d * (V[i] + V[i - 1]);
    double incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    double run = incl - tot;  // exclusive prefix of this lane's chunk
    if (i0 == 0 && i1 > 0) out[0] = 0.0;
    for (int i = max(i0, 1); i < i1; ++i) {
        run += half_d * (V[i] + V[i - 1]);
        out[i] = run;
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
haissinski_kernel(const Desc<T>* __restrict__ dd, double s_csr, double tol, int max_iter, double* __restrict__ rho_out,
                  double* __restrict__ gp_out, int* __restrict__ info)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Desc<T>& D = *dd;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
    const int n = D.n, M = D.M, H = M / 2;
    const double d = D.delta, L = 0.5 * d * (n - 1);
    double2* bufA = reinterpret_cast<double2*>(smem);
    double2* bufB = bufA + H;
    double2* tw = bufB + H;
    double2* zh = tw + H;  // H + 1 entries
    double* rho = reinterpret_cast<double*>(zh + H + 1);
    double* nw = rho + n;
    double* V = nw + n;
    double* red = V + n;
    volatile int* flag = reinterpret_cast<volatile int*>(red + 8);

    // twiddles exp(-2 pi i k/M) and the impedance table, in FP64
    for (int k = tid; k < H; k += nt) {
        double sv, cv;
        sincospi(-2.0 * k / M, &sv, &cv);
        tw[k] = make_double2(cv, sv);
    }
    for (int k = tid; k <= H; k += nt) zh[k] = make_double2(double(D.zhat[k].x), double(D.zhat[k].y));
    // start: the unit Gaussian profile, normalised to Delta sum rho = 1; the
    // p-profile of the state likewise
    for (int i = tid; i < n; i += nt) {
        const double q = -L + d * i;
        rho[i] = exp(-0.5 * q * q);
    }
    __syncthreads();
    if (warp == 0) {
        const double s = warp_fixed_sum<double>(rho, n);
        if (lane == 0) red[0] = s;
    }
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
        rho[i] /= d * red[0];
        if (gp_out) gp_out[i] = rho[i];  // same grid and shape in p
    }
    if (tid == 0) *flag = 0;
    __syncthreads();

    int it = 0;
    bool converged = false;
    while (it < max_iter && !converged) {
        ++it;
        // wake of rho (FP64): z_j = rho_2j + i rho_2j+1, zero-padded
        for (int j = tid; j < H; j += nt) {
            const int x = 2 * j;
            bufB[j] = make_double2(x < n ? rho[x] : 0.0, x + 1 < n ? rho[x + 1] : 0.0);
        }
        __syncthreads();
        double2* Z = fft_h<double, false>(bufB, bufA, bufB, tw, H, [] {});
        wake_pair_pass<double>(Z, tw, zh, H, d, nullptr, tid, nt);  // rho~ = Delta DFT(rho)
        __syncthreads();
        const double2* y = fft_h<double, true>(Z, Z == bufA ? bufB : bufA, Z, tw, H, [] {});
        for (int x = tid; x < n; x += nt) {
            const double2 v = y[x >> 1];
            V[x] = D.dkappa * ((x & 1) ? v.y : v.x);
        }
        __syncthreads();
        // Phi by the trapezoid rule, the exponent, its maximum
        if (warp == 0) warp_prefix_trapezoid(V, nw, n, 0.5 * d);
        __syncthreads();
        for (int i = tid; i < n; i += nt) {
            const double q = -L + d * i;
            nw[i] = -0.5 * q * q + s_csr * nw[i];
        }
        __syncthreads();
        if (warp == 0) {
            double m = -INFINITY;
            for (int i = lane; i < n; i += 32) m = fmax(m, nw[i]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) red[1] = m;
        }
        __syncthreads();
        for (int i = tid; i < n; i += nt) nw[i] = exp(nw[i] - red[1]);
        __syncthreads();
        if (warp == 0) {
            const double s = warp_fixed_sum<double>(nw, n);
            if (lane == 0) red[2] = s;
        }
        __syncthreads();
        // new profile, the change against the old one, the damped update
        for (int i = tid; i < n; i += nt) nw[i] /= d * red[2];
        __syncthreads();
        if (warp == 0) {
            double e = 0.0, mr = 0.0;
            for (int i = lane; i < n; i += 32) {
                e = fmax(e, fabs(nw[i] - rho[i]));
                mr = fmax(mr, rho[i]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                e = fmax(e, __shfl_xor_sync(0xffffffffu, e, o));
                mr = fmax(mr, __shfl_xor_sync(0xffffffffu, mr, o));
            }
            if (lane == 0) *flag = (e < tol * mr) ? 1 : (isfinite(e) ? 0 : 2);
        }
        __syncthreads();
        for (int i = tid; i < n; i += nt) rho[i] = 0.5 * rho[i] + 0.5 * nw[i];
        const int f = *flag;
        __syncthreads();
        if (f == 2) break;  // non-finite: give up
        converged = (f == 1);
    }
    for (int i = tid; i < n; i += nt) rho_out[i] = rho[i];
    if (tid == 0) {
        info[0] = it;
        info[1] = converged ? 1 : 0;
    }
}

// psi(x, y) = rho(x) g(y) into the simulation's current state buffer.
template <typename T>
__global__ void outer_state_kernel(const Desc<T>* __restrict__ dd, const double* __restrict__ rho,
                                   const double* __restrict__ g)
{
    const Desc<T>& D = *dd;
    T* psi = D.psi[D.st->parity];
    const int n = D.n, ld = D.ld;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x) {
        const int x = int(e / n), y = int(e % n);
        psi[(size_t)x * ld + y] = T(rho[x] * g[y]);
    }
}

}  // namespace vfps
