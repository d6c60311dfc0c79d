// Pointing (Sect. 3, the unlensed-direction formula, and the spin phase of
// Fig. 1), in FP64 on the device:
//   n' = cos(a) n + sin(a)/a (a_theta e_theta + a_phi e_phi),  a = |alpha|
//   beta  = atan2(a_phi, a_theta)      (direction of the geodesic at n)
//   t'    = -sin(a) n + cos(a) d       (its tangent at n', d = alpha / a)
//   beta' = atan2(t'.e_phi(n'), t'.e_theta(n'))
//   chi   = beta - beta', wrapped to (-pi, pi]; chi = 0 when a = 0.
#include <cuda_runtime.h>
#include <math.h>

#include "internal.h"

namespace gsl {
namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kPi = 3.141592653589793238462643383280;

__global__ void k_pointing(int64_t n, const double *__restrict__ theta, const double *__restrict__ phi,
                           const double *__restrict__ ath, const double *__restrict__ aph,
                           double *__restrict__ theta_out, double *__restrict__ phi_out, double *__restrict__ chi_out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double st, ct, sp, cp;
    sincos(theta[i], &st, &ct);
    sincos(phi[i], &sp, &cp);
    const double at = ath[i], ap = aph[i];
    const double a = hypot(at, ap);
    if (a == 0.0) {
        double p = fmod(phi[i], kTwoPi);
        if (p < 0.0) p += kTwoPi;
        if (p >= kTwoPi) p = 0.0;
        theta_out[i] = theta[i];
        phi_out[i] = p;
        if (chi_out) chi_out[i] = 0.0;
        return;
    }
    // n, e_theta, e_phi at the observed direction
    const double nx = st * cp, ny = st * sp, nz = ct;
    const double tx = ct * cp, ty = ct * sp, tz = -st;
    const double px = -sp, py = cp;
    const double ia = 1.0 / a;
    const double dx = (at * tx + ap * px) * ia, dy = (at * ty + ap * py) * ia, dz = at * tz * ia;
    double sa, ca;
    sincos(a, &sa, &ca);
    const double qx = ca * nx + sa * dx, qy = ca * ny + sa * dy, qz = ca * nz + sa * dz;  // n'
    const double ux = -sa * nx + ca * dx, uy = -sa * ny + ca * dy, uz = -sa * nz + ca * dz;  // t'
    const double rho = hypot(qx, qy);
    const double th2 = atan2(rho, qz);
    double ph2 = atan2(qy, qx);
    if (ph2 < 0.0) ph2 += kTwoPi;
    if (ph2 >= kTwoPi) ph2 -= kTwoPi;
    theta_out[i] = th2;
    phi_out[i] = ph2;
    if (chi_out) {
        // e_theta(n') = (cos th' cos ph', cos th' sin ph', -sin th'), e_phi(n') = (-sin ph', cos ph', 0)
        double cp2 = 1.0, sp2 = 0.0;
        if (rho > 0.0) { cp2 = qx / rho; sp2 = qy / rho; }
        const double ct2 = qz, st2 = rho;
        const double ut = ct2 * (ux * cp2 + uy * sp2) - st2 * uz;
        const double up = -sp2 * ux + cp2 * uy;
        double chi = atan2(ap, at) - atan2(up, ut);
        while (chi > kPi) chi -= kTwoPi;
        while (chi <= -kPi) chi += kTwoPi;
        chi_out[i] = chi;
    }
}

}  // namespace

cudaError_t launch_pointing(int64_t n, const double *theta, const double *phi, const double *ath, const double *aph,
                            double *theta_out, double *phi_out, double *chi_out, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int thr = 256;
    k_pointing<<<(unsigned)((n + thr - 1) / thr), thr, 0, st>>>(n, theta, phi, ath, aph, theta_out, phi_out, chi_out);
    return cudaGetLastError();
}

}  // namespace gsl
