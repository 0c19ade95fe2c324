// The local psi solves of the decomposition build on the GPU (build_gpu.cu).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "mmd_internal.h"

namespace mmd {

// psi values of every patch of one level, aligned with orows (the supports
// Omega_j, ascending rows per patch, offsets optr): the same problem as the
// host's localized_psi, solved by one block per patch on the current device.
// phi_of_row: phi value of every fine row.  Returns 0, 1 when a local matrix
// is not positive definite, or -1 on a CUDA failure (err says which).
int psi_solves_gpu(const HCSR& A, const std::vector<int32_t>& patch_of, const std::vector<double>& phi_of_row,
                   const std::vector<int32_t>& optr, const std::vector<int32_t>& orows, int64_t np,
                   std::vector<double>& psival, std::string& err);

}  // namespace mmd
