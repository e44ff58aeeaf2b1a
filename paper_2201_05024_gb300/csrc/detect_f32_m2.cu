// FP32 detection kernels for M = 2 antennas.
#define APSM_DETECT_M 2
#include "detect_f32_inst.cuh"
