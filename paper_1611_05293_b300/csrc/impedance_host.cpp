// impedance_host.cpp -- dimensionless CSR impedances tabulated on the host in
// FP64, once per vfps_set_impedance call (Sec. II.B of the paper).
//
//   free space:       Zhat(kappa) = 2 Gamma(2/3) 3^(-1/3) (sqrt(3)/2 + i/2) kappa^(1/3)
//   parallel plates:  Zhat(kappa) = 4 pi^2 2^(1/3) Pi^(2/3) kappa^(-1/3)
//                                   * sum_{p>=0} [Ai'(u_p) Ci'(u_p) + u_p Ai(u_p) Ci(u_p)],
//                     Ci = Ai - i Bi,  u_p = pi^2 (2p+1)^2 2^(-8/3) (Pi/kappa)^(4/3).
// Zhat is the paper's Z(n)/Z0 scaled by 2 (sigma_z/R)^(1/3) at n = kappa R/sigma_z,
// so that the kick per radian is dp = +S_csr V(q) dtheta with S_csr = I_n R^(1/3)/sigma_z^(4/3);
// Pi = R^(1/2) sigma_z / h^(3/2) with h half the distance g = 2h between the plates
// (the shielding parameter of the threshold law S_th ~ 0.5 + 0.12 Pi).
//
// Airy functions for x >= 0, written for this library:
//   x <= 2:  Maclaurin series Ai = c1 f - c2 g, Bi = sqrt3 (c1 f + c2 g);
//   x > 2:   Ai, Ai' from K_{1/3}, K_{2/3} of zeta = 2/3 x^(3/2) through the integral
//            K_nu(z) = int_0^inf exp(-z cosh t) cosh(nu t) dt (trapezoid rule, which
//            converges geometrically for this analytic integrand), scaled by exp(zeta);
//            Bi, Bi' by the series (x <= 8) or the large-x expansion (x > 8), scaled
//            by exp(-zeta);
//   x >= 25: only the combination Ai'Bi' + x Ai Bi is needed there and is taken
//            from its large-x expansion 3/(16 pi) x^(-5/2) (1 + 105/(32 x^3)
//            + 75075/(2048 x^6) + 56581525/(65536 x^9)), relative error < 1e-12;
//            Ai'^2 + x Ai^2 is below exp(-160) and is dropped.  Below 25 the
//            direct products lose about 3e-16 x^3 to cancellation (two O(sqrt x)
//            terms leave O(x^-5/2)).
#include <cmath>
#include <complex>
#include <vector>

namespace vfps {
namespace {

const double kPi = 3.14159265358979323846;

struct AiryScaled {
    double ai, aip;  // Ai, Ai' times exp(+zeta)
    double bi, bip;  // Bi, Bi' times exp(-zeta)
};

void airy_series(double x, double& ai, double& aip, double& bi, double& bip)
{
    const double c1 = 1.0 / (std::pow(3.0, 2.0 / 3.0) * std::tgamma(2.0 / 3.0));
    const double c2 = 1.0 / (std::pow(3.0, 1.0 / 3.0) * std::tgamma(1.0 / 3.0));
    const double x3 = x * x * x;
    double f = 1.0, fp = 0.0, g = x, gp = 1.0;
    double tf = 1.0, tg = x;
    for (int k = 1; k < 200; ++k) {
        tf *= x3 / ((3.0 * k - 1.0) * (3.0 * k));
        tg *= x3 / ((3.0 * k) * (3.0 * k + 1.0));
        f += tf;
        g += tg;
        // derivative terms: d/dx x^(3k) = 3k x^(3k-1)
        if (x > 0.0) {
            fp += tf * (3.0 * k) / x;
            gp += tg * (3.0 * k + 1.0) / x;
        }
        if (tf < 1e-18 * f && tg < 1e-18 * std::fabs(g) + 1e-300) break;
    }
    if (x == 0.0) { fp = 0.0; gp = 1.0; }
    ai = c1 * f - c2 * g;
    aip = c1 * fp - c2 * gp;
    bi = std::sqrt(3.0) * (c1 * f + c2 * g);
    bip = std::sqrt(3.0) * (c1 * fp + c2 * gp);
}

// exp(z) K_nu(z) = int_0^inf exp(-z (cosh t - 1)) cosh(nu t) dt.  The
// integrand peaks at t = 0 with width ~ 1/sqrt(z); a step of half that width
// puts the trapezoid error near exp(-8 pi^2).
double k_scaled(double nu, double z)
{
    const double hstep = std::fmin(0.1, 0.5 / std::sqrt(z));
    double s = 0.5;  // t = 0 term: cosh(0) = 1, weight 1/2
    for (int k = 1; k < 100000; ++k) {
        double t = k * hstep;
        double e = z * (std::cosh(t) - 1.0);
        if (e > 745.0) break;
        double term = std::exp(-e) * std::cosh(nu * t);
        s += term;
        if (term < 1e-19 * s) break;
    }
    return hstep * s;
}

AiryScaled airy_scaled(double x)
{
    AiryScaled r{};
    double zeta = (2.0 / 3.0) * x * std::sqrt(x);
    if (x <= 2.0) {
        double ai, aip, bi, bip;
        airy_series(x, ai, aip, bi, bip);
        double ez = std::exp(zeta);
        r.ai = ai * ez;
        r.aip = aip * ez;
        r.bi = bi / ez;
        r.bip = bip / ez;
        return r;
    }
    r.ai = std::sqrt(x / 3.0) / kPi * k_scaled(1.0 / 3.0, zeta);
    r.aip = -x / (kPi * std::sqrt(3.0)) * k_scaled(2.0 / 3.0, zeta);
    if (x <= 8.0) {
        double ai, aip, bi, bip;
        airy_series(x, ai, aip, bi, bip);
        double ez = std::exp(zeta);
        r.bi = bi / ez;
        r.bip = bip / ez;
    } else {
        // DLMF 9.7.7-9.7.8 coefficients u_k, v_k
        double u = 1.0, su = 1.0, sv = 1.0, zk = 1.0, prev = 1e300;
        for (int k = 1; k < 60; ++k) {
            u *= (6.0 * k - 5.0) * (6.0 * k - 3.0) * (6.0 * k - 1.0) / ((2.0 * k - 1.0) * 216.0 * k);
            double v = -(6.0 * k + 1.0) / (6.0 * k - 1.0) * u;
            zk *= zeta;
            double tu = u / zk, tv = v / zk;
            if (std::fabs(tu) > prev) break;  // asymptotic series: stop at the smallest term
            prev = std::fabs(tu);
            su += tu;
            sv += tv;
            if (std::fabs(tu) < 1e-17) break;
        }
        double x14 = std::pow(x, 0.25);
        r.bi = su / (std::sqrt(kPi) * x14);
        r.bip = sv * x14 / std::sqrt(kPi);
    }
    return r;
}

// F(u) = Ai'(u) Ci'(u) + u Ai(u) Ci(u) with Ci = Ai - i Bi
std::complex<double> f_term(double u)
{
    if (u >= 25.0) {
        double v = 1.0 / (u * u * u);
        double g = 3.0 / (16.0 * kPi) * std::pow(u, -2.5) *
                   (1.0 + v * (105.0 / 32.0 + v * (75075.0 / 2048.0 + v * (56581525.0 / 65536.0))));
        return {0.0, -g};
    }
    AiryScaled a = airy_scaled(u);
    double zeta = (2.0 / 3.0) * u * std::sqrt(u);
    double damp = std::exp(-2.0 * zeta);
    double re = (a.aip * a.aip + u * a.ai * a.ai) * damp;
    double im = -(a.aip * a.bip + u * a.ai * a.bi);
    return {re, im};
}

}  // namespace

std::complex<double> zhat_free_space(double kappa)
{
    const double c = 2.0 * std::tgamma(2.0 / 3.0) * std::pow(3.0, -1.0 / 3.0);
    double k13 = std::cbrt(kappa);
    return {c * std::sqrt(3.0) / 2.0 * k13, c * 0.5 * k13};
}

std::complex<double> zhat_parallel_plates(double kappa, double Pi)
{
    if (!(kappa > 0.0)) return {0.0, 0.0};
    const double a = kPi * kPi * std::pow(2.0, -8.0 / 3.0) * std::pow(Pi / kappa, 4.0 / 3.0);
    std::complex<double> s{0.0, 0.0};
    // terms fall off like (2p+1)^-5 once u_p is large; sum until negligible
    std::vector<std::complex<double>> terms;
    for (long p = 0; p < 4000000; ++p) {
        double sp = 2.0 * p + 1.0;
        double u = a * sp * sp;
        std::complex<double> f = f_term(u);
        terms.push_back(f);
        s += f;
        if (u >= 25.0 && std::abs(f) < 1e-18 * std::abs(s)) {
            // remainder: sum_{q>p} (2q+1)^-5 ~ int_{p+1/2}^inf (2q+1)^-5 dq
            double rem = 3.0 / (16.0 * kPi) * std::pow(a, -2.5) * std::pow(2.0 * p + 2.0, -4.0) / 8.0;
            terms.push_back({0.0, -rem});
            break;
        }
    }
    // re-sum from the smallest terms up
    std::complex<double> acc{0.0, 0.0};
    for (size_t i = terms.size(); i-- > 0;) acc += terms[i];
    double pref = 4.0 * kPi * kPi * std::cbrt(2.0) * std::pow(Pi, 2.0 / 3.0) * std::pow(kappa, -1.0 / 3.0);
    return pref * acc;
}

// Table on the FFT grid kappa_k = 2 pi k/(M Delta), k = 0..M/2.
// model 0 none, 1 free space, 2 parallel plates.
void impedance_table(int model, int M, double delta, double Pi, std::vector<std::complex<double>>& z)
{
    int K = M / 2;
    z.assign(K + 1, {0.0, 0.0});
    if (model == 0) return;
    double dk = 2.0 * kPi / (M * delta);
    for (int k = 1; k <= K; ++k) {
        double kap = k * dk;
        z[k] = (model == 1) ? zhat_free_space(kap) : zhat_parallel_plates(kap, Pi);
    }
}

}  // namespace vfps
