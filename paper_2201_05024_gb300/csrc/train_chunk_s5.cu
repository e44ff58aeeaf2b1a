// Phase-B training kernels for S = 5 live-range warps.
#define APSM_CHUNK_S 5
#include "train_chunk_inst.cuh"
