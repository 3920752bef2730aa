// Step-kernel instances for BF16 storage of the (f, g) pairs and FP32 storage of h.
#include "lbm_launch.h"

namespace lbm {

LBM_DEFINE_STORAGE(bf16fg, kBF16FG)

}  // namespace lbm
