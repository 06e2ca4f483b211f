// Chunk kernels of the batch: 128 chains per CTA, sweep loop unrolled 2x.
#include "batch_chunks.cuh"

namespace xzzx {
namespace batch {
XZZX_CHUNK_VARIANT(128, 2)
}  // namespace batch
}  // namespace xzzx
