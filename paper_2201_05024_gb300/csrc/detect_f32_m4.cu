// FP32 detection kernels for M = 4 antennas.
#define APSM_DETECT_M 4
#include "detect_f32_inst.cuh"
