// Step-kernel instances for FP16 storage of the (f, g) pairs and FP32 storage of h.
#include "lbm_launch.h"

namespace lbm {

LBM_DEFINE_STORAGE(fp16fg, kFP16FG)

}  // namespace lbm
