// FP32 sweeps on FP64 state: the sweeps read the FP32 copy of the state, the
// boundary solve and the state update run in FP64.
#include "sweep_launch.h"

namespace molt {
MOLT_DEFINE_LAUNCH
MOLT_INST(float, float, double, false, EPI_STORE)
MOLT_INST(float, float, double, false, EPI_ACC_SET)
MOLT_INST(float, float, double, false, EPI_ACC_ADD)
MOLT_INST(float, float, double, false, EPI_HEAT_FINAL)
MOLT_INST(float, float, double, false, EPI_WAVE_FINAL)
MOLT_INST(float, double, double, false, EPI_STORE)
MOLT_INST(float, double, double, true, EPI_STORE)
}  // namespace molt
