// Phase-B training kernels for S = 5 live-range warps, extended instantiations.
#define APSM_CHUNK_S 5
#define APSM_CHUNK_EXT 1
#include "train_chunk_inst.cuh"
