// Phase-B training kernels for S = 2 live-range warps.
#define APSM_CHUNK_S 2
#include "train_chunk_inst.cuh"
