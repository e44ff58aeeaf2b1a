// Tensor-core detection kernels for M = 8 antennas.
#define APSM_TC_M 8
#include "detect_tc_inst.cuh"
