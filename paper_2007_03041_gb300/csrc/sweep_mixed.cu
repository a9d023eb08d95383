// FP32 sweeps on FP64 state: the sweeps read the FP32 copy of the state, the
// boundary solve and the state update run in FP64.
#include "sweep_launch.h"

namespace molt {
MOLT_DEFINE_LAUNCH
MOLT_INST(float, float, double, JQ_LINEAR, EPI_STORE)
MOLT_INST(float, float, double, JQ_LINEAR, EPI_ACC_SET)
MOLT_INST(float, float, double, JQ_LINEAR, EPI_ACC_ADD)
MOLT_INST(float, float, double, JQ_LINEAR, EPI_HEAT_FINAL)
MOLT_INST(float, float, double, JQ_LINEAR, EPI_WAVE_FINAL)
MOLT_INST(float, double, double, JQ_LINEAR, EPI_STORE)
MOLT_INST(float, double, double, JQ_WENOZ, EPI_STORE)
}  // namespace molt
