// BLOCK-scope rows kernels for Plain<OrU>, Plain<XorU>, Plain<MinI> (see reduce_block_rows.cuh).
#define COX_BLOCK_ROWS_IMPL
#include "reduce_block_rows.cuh"

namespace cox {
template cox_status block_rows_launch<Plain<OrU>>(int, int, const void*, void*, float*, int64_t, cudaStream_t);
template cox_status block_rows_launch<Plain<XorU>>(int, int, const void*, void*, float*, int64_t, cudaStream_t);
template cox_status block_rows_launch<Plain<MinI>>(int, int, const void*, void*, float*, int64_t, cudaStream_t);

}  // namespace cox
