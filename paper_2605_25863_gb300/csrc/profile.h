// profile.h -- optional per-kernel-class timing of the library's launches.
// When enabled, each launch is bracketed by CUDA events recorded on its own
// stream; totals are read back by linac_profile_read().  Launches are always
// counted (linac_launch_count()).
#pragma once
#include <cuda_runtime.h>

namespace linac {

enum ProfClass {
    PROF_INIT = 0, PROF_PANEL, PROF_GATHER_F, PROF_GATHER_W, PROF_INVERSE, PROF_TRSM, PROF_MOVE,
    PROF_UPDATE_PLAIN, PROF_UPDATE_LIMB, PROF_LIMB_SPLIT, PROF_FINISH, PROF_BATCHED, PROF_SOLVE_PACK,
    PROF_SOLVE_EXTRACT, PROF_VALIDATE, PROF_PATTERN, PROF_MATMUL, PROF_LOAD_MATRIX, PROF_DERIVED, PROF_U64_PANEL, PROF_U64_UPDATE,
    PROF_UPDATE_CRT, PROF_CRT_SPLIT, PROF_HOST_COPY, PROF_LUP, PROF_UPDATE_HYBRID, PROF_NCLASSES
};

const char* prof_name(int cls);
void prof_begin(cudaStream_t s, int cls);
void prof_end(cudaStream_t s, int cls);

struct ProfScope {
    cudaStream_t s;
    int cls;
    ProfScope(cudaStream_t s_, int c) : s(s_), cls(c) { prof_begin(s, cls); }
    ~ProfScope() { prof_end(s, cls); }
};

}  // namespace linac
