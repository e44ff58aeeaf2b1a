// FP32 detection kernels for M = 32 antennas.
#define APSM_DETECT_M 32
#include "detect_f32_inst.cuh"
