// Kernel instances for rows of 12 edges, compiled apart from the rest so
// that the build runs them in parallel: the mixed-batch kernels of each shape
// class (mixed_core.cuh) and the resident kernels with fixed plane sizes
// (resident_core.cuh).
#include "mixed_core.cuh"

namespace ldpc {

MixedFn mixed_fn_rows12(bool fp16, bool syn, int pl) { return mixed_pick<12, 4>(fp16, syn, pl); }

KernelFn resident_fixed_rows12(int pl, bool syn) { return resident_fixed_pick<12, 4>(pl, syn); }

}  // namespace ldpc
