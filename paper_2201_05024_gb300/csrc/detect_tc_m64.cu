// Tensor-core detection kernels for M = 64 antennas.
#define APSM_TC_M 64
#include "detect_tc_inst.cuh"
