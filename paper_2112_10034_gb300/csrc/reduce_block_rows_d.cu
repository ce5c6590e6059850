// BLOCK-scope rows kernels for Plain<MaxI>, Plain<MinU>, Plain<MaxU> (see reduce_block_rows.cuh).
#define COX_BLOCK_ROWS_IMPL
#include "reduce_block_rows.cuh"

namespace cox {
template cox_status block_rows_launch<Plain<MaxI>>(int, int, const void*, void*, float*, int64_t, cudaStream_t);
template cox_status block_rows_launch<Plain<MinU>>(int, int, const void*, void*, float*, int64_t, cudaStream_t);
template cox_status block_rows_launch<Plain<MaxU>>(int, int, const void*, void*, float*, int64_t, cudaStream_t);

}  // namespace cox
