// FP32 detection kernels for M = 64 antennas.
#define APSM_DETECT_M 64
#include "detect_f32_inst.cuh"
