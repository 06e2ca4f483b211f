// Chunk kernels of the batch: 256 chains per CTA, sweep loop unrolled 1x.
#include "batch_chunks.cuh"

namespace xzzx {
namespace batch {
XZZX_CHUNK_VARIANT(256, 1)
}  // namespace batch
}  // namespace xzzx
