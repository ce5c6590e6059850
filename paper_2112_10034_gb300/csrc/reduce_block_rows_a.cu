// BLOCK-scope rows kernels for Comp, Plain<AddF>, Plain<MinF> (see reduce_block_rows.cuh).
#define COX_BLOCK_ROWS_IMPL
#include "reduce_block_rows.cuh"

namespace cox {
template cox_status block_rows_launch<Comp>(int, int, const void*, void*, float*, int64_t, cudaStream_t);
template cox_status block_rows_launch<Plain<AddF>>(int, int, const void*, void*, float*, int64_t, cudaStream_t);
template cox_status block_rows_launch<Plain<MinF>>(int, int, const void*, void*, float*, int64_t, cudaStream_t);

}  // namespace cox
