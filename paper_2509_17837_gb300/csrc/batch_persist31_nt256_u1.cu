// Persistent annealing kernel of the batch for distances up to 31, 256 chains
// per CTA, sweep loop unrolled 1x.
#include "batch_persist.cuh"

namespace xzzx {
namespace batch {
XZZX_PERSIST_VARIANT(31, 256, 1)
}  // namespace batch
}  // namespace xzzx
