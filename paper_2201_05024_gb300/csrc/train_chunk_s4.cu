// Phase-B training kernels for S = 4 live-range warps.
#define APSM_CHUNK_S 4
#include "train_chunk_inst.cuh"
