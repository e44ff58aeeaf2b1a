// FP32 detection kernels for M = 16 antennas.
#define APSM_DETECT_M 16
#include "detect_f32_inst.cuh"
