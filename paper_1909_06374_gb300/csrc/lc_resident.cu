// lc_resident.cu -- fused on-chip iteration for short curves (filled in by the
// resident kernel; until then every class uses the multi-kernel path).
#include "lc_internal.h"

namespace lc {

bool resident_supported(const Plan&, uint32_t) { return false; }

void launch_resident(const Plan&, const ClassInfo&, uint32_t, cudaStream_t, uint64_t*) {}

}  // namespace lc
