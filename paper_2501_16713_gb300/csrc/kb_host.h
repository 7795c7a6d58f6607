// Host FP64 math of the interpolation kernel (plan time only).
#pragma once

#include "common.cuh"

namespace nrs {

// I0(z) - 1 by its power series (summed from k = 1, no cancellation).
double bessel_i0m1(double z);
// Beatty et al.'s Kaiser-Bessel shape parameter for width W, oversampling osf.
double beatty_beta(int width, double osf);
// Edge-subtracted Kaiser-Bessel kernel c(u), zero for |u| >= W/2.
double kb_kernel(double u, int width, double beta);
// Its Fourier transform C(nu) in closed form.
double kb_kernel_ft(double nu, int width, double beta);
// Fit the per-tap FP32 polynomials; returns max |p - c| / c(0) of the FP32
// evaluation on a fine grid.
double fit_kernel_polys(int width, double beta, KernelCoefs* out);

}  // namespace nrs
