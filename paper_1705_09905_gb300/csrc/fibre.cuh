// fibre.cuh -- the fibre tensor of an SpTTM handle (fibre.cu), shared by the
// by-fibre SpTTMc plan and the CP-ALS fibre reuse.
#pragma once

#include "internal.cuh"

namespace fcx {

// The fibre tensor of a 3-way SpTTM handle along mode b: one nonzero of value
// 1 per fibre f, at (k0, k1, f), where (k0, k1) is the fibre's index-mode
// tuple (index modes ascending).  Built as an F-COO for SpMTTKRP on `mode`
// (0: rows k0, product modes k1 and f; 1: rows k1, product modes k0 and f),
// so that Eq. 6 or Eq. 4 over it, with the fibre sums of Eq. 3 as the
// factor of the third mode, regroups the same sums over the original
// nonzeros by fibre.  Synchronous (fcoo_build).
int fibre_tensor_build(const fcoo_t *Xttm, int mode, int threadlen, cudaStream_t s, fcoo_t **out);

}  // namespace fcx
