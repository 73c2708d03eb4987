// mhd_fp64.cu -- step pipelines instantiated for one precision (double,double,double).
#include "mhd_engine.cuh"

mhd_step_fn mhd_pick_fp64(int integ, int recon, int solver, cudaError_t* attr)
{
    return mhd::pick_step<double,double,double>(integ, recon, solver, attr);
}
