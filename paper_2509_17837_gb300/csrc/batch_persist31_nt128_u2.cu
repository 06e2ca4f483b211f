// Persistent annealing kernel of the batch for distances up to 31, 128 chains
// per CTA, sweep loop unrolled 2x.
#include "batch_persist.cuh"

namespace xzzx {
namespace batch {
XZZX_PERSIST_VARIANT(31, 128, 2)
}  // namespace batch
}  // namespace xzzx
