// gp_output.h -- launcher of the density-profile kernels (k_output.cu).
#pragma once

#include "gp_internal.h"

namespace gpcn {

// Integrated density profiles rho_x, rho_y, rho_z of a.psi (times the square
// of *a.scale) into out[0 .. nx+ny+nz): x nodes, then y, then z.  scratch
// holds profile_scratch_doubles(a) doubles of device memory.
size_t profile_scratch_doubles(const FieldArgs &a);
cudaError_t launch_density_profiles(Prec p, bool cplx, const FieldArgs &a, double *scratch, double *out,
                                    cudaStream_t s);

}  // namespace gpcn
