// Step-kernel instances for FP16 population storage.
#include "lbm_launch.h"

namespace lbm {

LBM_DEFINE_STORAGE(fp16, kFP16)

}  // namespace lbm
