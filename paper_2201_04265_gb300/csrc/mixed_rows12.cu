// K6 mixed-batch kernels for rows of 12 edges (mixed_core.cuh).
#include "mixed_core.cuh"

namespace ldpc {

MixedFn mixed_fn_rows12(bool fp16, bool syn, int pl) { return mixed_pick<12, 4>(fp16, syn, pl); }

}  // namespace ldpc
