// Spectrum from the autocorrelation function (Sec. 3.1): the damped Fourier
// transform of C(t) = <psi(0)|psi(t)> sampled at t_k = k dt,
//
//   I(E) = 1/(pi hbar) Re sum_k w_k C(t_k) exp(+i E t_k / hbar) exp(-t_k / tau),
//
// w_k = dt (dt/2 at both ends: the trapezoidal rule of the half-axis
// integral; C(-t) = conj C(t) makes twice its real part the transform over
// the whole axis). One CTA per energy, FP64, the phases from sincos of the
// exact argument (no accumulated rotation).
#include "common.h"

namespace vb {
namespace {

constexpr double HBAR = 0.6582119569;  // eV fs
constexpr int SPEC_THREADS = 256;

__global__ void __launch_bounds__(SPEC_THREADS) spectrum_kernel(const cd *__restrict__ c, int n_t, double dt,
                                                                 double inv_tau, const double *__restrict__ energies,
                                                                 double *__restrict__ out) {
  const double e = energies[blockIdx.x];
  double acc = 0.0;
  for (int k = threadIdx.x; k < n_t; k += SPEC_THREADS) {
    const double t = dt * (double)k;
    double sn, cs;
    sincos(e * t / HBAR, &sn, &cs);
    const double w = (k == 0 || k == n_t - 1) ? 0.5 * dt : dt;
    const cd z = c[k];
    // Re[(z.x + i z.y)(cs + i sn)] = z.x cs - z.y sn
    acc += w * exp(-t * inv_tau) * (z.x * cs - z.y * sn);
  }
  __shared__ double red[SPEC_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < SPEC_THREADS / 32 ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) out[blockIdx.x] = v / (M_PI * HBAR);
  }
}

}  // namespace
}  // namespace vb

extern "C" vb_status vb_spectrum(const double *c_t, int n_t, double dt_fs, double tau_fs, const double *energies,
                                 int n_e, double *out, void *stream) {
  using namespace vb;
  if (n_t < 1 || n_e < 0 || !c_t || (n_e > 0 && (!energies || !out)) || !(dt_fs > 0) || !(tau_fs > 0))
    return fail(VB_EINVAL, "vb_spectrum: bad argument");
  if (n_e == 0) return VB_OK;
  spectrum_kernel<<<n_e, SPEC_THREADS, 0, (cudaStream_t)stream>>>(reinterpret_cast<const cd *>(c_t), n_t, dt_fs,
                                                                  1.0 / tau_fs, energies, out);
  VB_CHECK_LAUNCH();
  return VB_OK;
}
