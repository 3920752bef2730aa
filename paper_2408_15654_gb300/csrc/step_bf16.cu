// Step-kernel instances for BF16 population storage.
#include "lbm_launch.h"

namespace lbm {

LBM_DEFINE_STORAGE(bf16, kBF16)

}  // namespace lbm
