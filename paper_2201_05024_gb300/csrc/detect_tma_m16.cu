// TMA-staged tensor-core detection kernels for M = 16 antennas.
#define APSM_TMA_M 16
#include "detect_tma_inst.cuh"
