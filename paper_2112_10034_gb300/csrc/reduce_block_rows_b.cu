// BLOCK-scope rows kernels for Plain<MaxF>, Plain<AddU>, Plain<AndU> (see reduce_block_rows.cuh).
#define COX_BLOCK_ROWS_IMPL
#include "reduce_block_rows.cuh"

namespace cox {
template cox_status block_rows_launch<Plain<MaxF>>(int, int, const void*, void*, float*, int64_t, cudaStream_t);
template cox_status block_rows_launch<Plain<AddU>>(int, int, const void*, void*, float*, int64_t, cudaStream_t);
template cox_status block_rows_launch<Plain<AndU>>(int, int, const void*, void*, float*, int64_t, cudaStream_t);

}  // namespace cox
