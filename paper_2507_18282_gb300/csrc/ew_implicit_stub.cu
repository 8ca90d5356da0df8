#include "ew_internal.h"
namespace ew {
ew_status implicit_wave_solve_any(ew_grid*, const FilterPlan&, const ew_filter_params*, const void*, void*, int,
                                  cudaStream_t) {
    return set_error(EW_EUNSUPPORTED, "implicit scheme not built");
}
}  // namespace ew
