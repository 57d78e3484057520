// Host helpers shared by the single-instance, batched and serving code.
#pragma once

#include "raster_device.cuh"

namespace raster {

// Split the scale s into odd significand and exponent for the integer
// projection; *wide is set when the significand needs a 128-bit product.
// Returns RASTER_E_ARG unless s is a normal positive double.
int make_proj_params(double scale, ProjParams* pp, bool* wide);

// s = 10^precision: the exact double for integer precisions 0..22, else the
// host C library's pow(10, precision).
double scale_of_precision(double precision);

// Count k kernel launches issued by this library (diagnostics).
void note_launch(unsigned long long k = 1);

// Bounds of the device loops chosen for tests of the failure paths
// (raster_set_test_limits); negative means the library's own bound.  Read
// when a handle, batch or served request is created.
struct TestLimits {
    int probe;   // most slots one insertion probes
    int unions;  // most steps of one union-find join
};
TestLimits test_limits();

}  // namespace raster
