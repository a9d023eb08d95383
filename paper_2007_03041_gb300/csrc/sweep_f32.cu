// FP32 sweeps on FP32 state.
#include "sweep_launch.h"

namespace molt {
MOLT_DEFINE_LAUNCH
MOLT_INST(float, float, float, JQ_LINEAR, EPI_STORE)
MOLT_INST(float, float, float, JQ_LINEAR, EPI_ACC_SET)
MOLT_INST(float, float, float, JQ_LINEAR, EPI_ACC_ADD)
MOLT_INST(float, float, float, JQ_LINEAR, EPI_HEAT_FINAL)
MOLT_INST(float, float, float, JQ_LINEAR, EPI_WAVE_FINAL)
MOLT_INST(float, float, float, JQ_LINEAR, EPI_HJ_X)
MOLT_INST(float, float, float, JQ_LINEAR, EPI_HJ_Y)
MOLT_INST(float, float, float, JQ_WENOZ, EPI_STORE)
MOLT_INST(float, float, float, JQ_WENOZ, EPI_HJ_X)
MOLT_INST(float, float, float, JQ_WENOZ, EPI_HJ_Y)
MOLT_INST(float, float, float, JQ_LEARNED, EPI_STORE)
MOLT_INST(float, float, float, JQ_LEARNED, EPI_HJ_X)
MOLT_INST(float, float, float, JQ_LEARNED, EPI_HJ_Y)
}  // namespace molt
