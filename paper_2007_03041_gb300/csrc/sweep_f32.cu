// FP32 sweeps on FP32 state.
#include "sweep_launch.h"

namespace molt {
MOLT_DEFINE_LAUNCH
MOLT_INST(float, float, float, false, EPI_STORE)
MOLT_INST(float, float, float, false, EPI_ACC_SET)
MOLT_INST(float, float, float, false, EPI_ACC_ADD)
MOLT_INST(float, float, float, false, EPI_HEAT_FINAL)
MOLT_INST(float, float, float, false, EPI_WAVE_FINAL)
MOLT_INST(float, float, float, false, EPI_HJ_X)
MOLT_INST(float, float, float, false, EPI_HJ_Y)
MOLT_INST(float, float, float, true, EPI_STORE)
MOLT_INST(float, float, float, true, EPI_HJ_X)
MOLT_INST(float, float, float, true, EPI_HJ_Y)
}  // namespace molt
