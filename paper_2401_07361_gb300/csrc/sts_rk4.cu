// Classical fourth-order Runge-Kutta step (Sec. 4: the particle system of Sec. 2 is
// advanced with RK4) for the state (x_i, zeta_i) with dx_i/dt = u_i and
// dzeta_i/dt = -2 Omega dz_i/dt = -2 Omega u_z,i (Sec. 2, absolute vorticity zeta + 2 Omega z
// is carried by each particle).  Stage points and the new positions are projected back to
// the unit sphere, x / |x|.  All in FP64, one fused pass per stage.
#include "sts_internal.cuh"

namespace sts {
namespace {

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ void project(double& x, double& y, double& z)
{
    const double r = sqrt((x * x + y * y) + z * z);
    x /= r;
    y /= r;
    z /= r;
}

// ksum (+)= b k; xs = proj(x0 + cdt k); zs = z0 + cdt (-2 Omega k_z)
__global__ void k_stage(const double* __restrict__ x0, const double* __restrict__ z0,
                        const double* __restrict__ k, double cdt, double Omega,
                        double* __restrict__ xs, double* __restrict__ zs, double* __restrict__ ksum,
                        double b, int first, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double kx = k[3 * i], ky = k[3 * i + 1], kz = k[3 * i + 2];
    if (first) {
        ksum[3 * i] = b * kx;
        ksum[3 * i + 1] = b * ky;
        ksum[3 * i + 2] = b * kz;
    } else {
        ksum[3 * i] += b * kx;
        ksum[3 * i + 1] += b * ky;
        ksum[3 * i + 2] += b * kz;
    }
    double x = x0[3 * i] + cdt * kx, y = x0[3 * i + 1] + cdt * ky, z = x0[3 * i + 2] + cdt * kz;
    project(x, y, z);
    xs[3 * i] = x;
    xs[3 * i + 1] = y;
    xs[3 * i + 2] = z;
    zs[i] = z0[i] + cdt * (-2.0 * Omega * kz);
}

// x = proj(x0 + dt/6 (ksum + k4)); z = z0 + dt/6 (-2 Omega (ksum + k4)_z)
__global__ void k_final(double* __restrict__ x, double* __restrict__ z, const double* __restrict__ x0,
                        const double* __restrict__ z0, const double* __restrict__ ksum,
                        const double* __restrict__ k4, double dt, double Omega, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double sx = ksum[3 * i] + k4[3 * i], sy = ksum[3 * i + 1] + k4[3 * i + 1];
    const double sz = ksum[3 * i + 2] + k4[3 * i + 2];
    const double h = dt / 6.0;
    double a = x0[3 * i] + h * sx, b = x0[3 * i + 1] + h * sy, c = x0[3 * i + 2] + h * sz;
    project(a, b, c);
    x[3 * i] = a;
    x[3 * i + 1] = b;
    x[3 * i + 2] = c;
    z[i] = z0[i] + h * (-2.0 * Omega * sz);
}

// Source vorticity of the forced system (Sec. 4.4): zf = zs - c B(theta) cos(k phi), with
// c = amplitude k^2 A(t) from the host, theta the latitude, phi the longitude of the stage
// point, B = r exp(1 - r), r = tan^2 theta1 / tan^2 theta north of the equator, 0 south.
__global__ void k_forced_source(const double* __restrict__ xs, const double* __restrict__ zs, int64_t n,
                                double c, int k, double tan2t1, double* __restrict__ zf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = xs[3 * i], y = xs[3 * i + 1], z = xs[3 * i + 2];
    const double lat = asin(fmin(1.0, fmax(-1.0, z)));
    double F = 0.0;
    if (lat > 0.0 && c != 0.0) {
        const double t = tan(lat);
        const double r = tan2t1 / (t * t);
        F = c * (r * exp(1.0 - r)) * cos(k * atan2(y, x));
    }
    zf[i] = zs[i] - F;
}

}  // namespace

// A(t) of Sec. 4.4: half-cosine ramps of length Tp at both ends of [0, Tf], 1 between.
double forcing_ramp(double t, double Tp, double Tf)
{
    const double pi = 3.14159265358979323846;
    if (t < 0.0 || t >= Tf) return 0.0;
    if (t < Tp) return (1.0 - cos(t / Tp * pi)) / 2.0;
    if (t < Tf - Tp) return 1.0;
    return (1.0 - cos(pi + (t - Tf + Tp) / Tp * pi)) / 2.0;
}

void forced_source(const double* xs, const double* zs, int64_t n, const sts_forcing* f, double t, double* zf,
                   cudaStream_t s)
{
    const double c = f->amplitude * (double)f->k * (double)f->k * forcing_ramp(t, f->Tp, f->Tf);
    const double t1 = tan(f->theta1);
    if (n > 0)
        (k_forced_source<<<blocks(n, 256), 256, 0, s>>>(xs, zs, n, c, f->k, t1 * t1, zf), note_launch());
}

void rk4_stage(const double* x0, const double* z0, const double* k, double cdt, double Omega,
               double* xs, double* zs, double* ksum, double b, int first, int64_t n, cudaStream_t s)
{
    if (n > 0) (k_stage<<<blocks(n, 256), 256, 0, s>>>(x0, z0, k, cdt, Omega, xs, zs, ksum, b, first, n), note_launch());
}

void rk4_final(double* x, double* z, const double* x0, const double* z0, const double* ksum,
               const double* k4, double dt, double Omega, int64_t n, cudaStream_t s)
{
    if (n > 0) (k_final<<<blocks(n, 256), 256, 0, s>>>(x, z, x0, z0, ksum, k4, dt, Omega, n), note_launch());
}

}  // namespace sts
