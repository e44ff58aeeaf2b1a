// Tensor-core detection kernels for M = 16 antennas.
#define APSM_TC_M 16
#include "detect_tc_inst.cuh"
