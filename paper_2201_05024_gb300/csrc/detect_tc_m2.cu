// Tensor-core detection kernels for M = 2 antennas.
#define APSM_TC_M 2
#include "detect_tc_inst.cuh"
