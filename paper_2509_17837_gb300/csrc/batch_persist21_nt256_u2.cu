// Persistent annealing kernel of the batch for distances up to 21, 256 chains
// per CTA, sweep loop unrolled 2x.
#include "batch_persist.cuh"

namespace xzzx {
namespace batch {
XZZX_PERSIST_VARIANT(21, 256, 2)
}  // namespace batch
}  // namespace xzzx
