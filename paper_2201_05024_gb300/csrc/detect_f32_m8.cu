// FP32 detection kernels for M = 8 antennas.
#define APSM_DETECT_M 8
#include "detect_f32_inst.cuh"
