// Device-driven runs of a single system.  A conditional node between two MD
// steps of a CUDA graph costs ~7.7 us on GB300 even when it is not taken,
// about a tenth of a 1M-bead step.  Instead, prx_run launches a device graph
// holding one step (the step kernel(s), then k_dg_next), and k_dg_next
// decides on the device what follows: the rebuild graph when a particle
// moved more than skin/2, the reaction graph after every Theta-th step, then
// the step graph itself until the run's steps are done, each as a tail
// launch (tail launches run in the order they were made, each after the
// previous one and the launching graph completed; the host stream sees the
// whole chain as the one graph it launched).  This file alone is compiled
// with relocatable device code (device-side graph launches need it); the
// step kernel itself is not.
#include <cuda_runtime.h>

#include "prx_internal.cuh"

namespace prx {

namespace {

__global__ void k_dg_arm(Ctl* ctl, unsigned long long steps, unsigned long long rebuild,
                         unsigned long long react) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->steps_left = steps;
    ctl->dg_rebuild = rebuild;
    ctl->dg_react = react;
  }
}

// After step ctl->step (written by the step kernel's last warp): what runs
// next.  A failed launch sets PRX_ECUDA and ends the chain.
__global__ void k_dg_next(Ctl* ctl, int has_rx, unsigned int theta) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned long long step = ctl->step;
  bool ok = true;
  if (ctl->rebin_flag)
    ok = cudaGraphLaunch((cudaGraphExec_t)ctl->dg_rebuild, cudaStreamGraphTailLaunch) == cudaSuccess;
  if (ok && has_rx && step % theta == 0)
    ok = cudaGraphLaunch((cudaGraphExec_t)ctl->dg_react, cudaStreamGraphTailLaunch) == cudaSuccess;
  if (ok && ctl->steps_left > 1ull) {
    ctl->steps_left -= 1ull;
    ok = cudaGraphLaunch(cudaGetCurrentGraphExec(), cudaStreamGraphTailLaunch) == cudaSuccess;
  } else {
    ctl->steps_left = 0ull;
  }
  if (!ok) atomicCAS(&ctl->status, 0, PRX_ECUDA);
}

}  // namespace

void launch_dg_arm(const Sys& S, cudaStream_t st, unsigned long long steps,
                   unsigned long long rebuild, unsigned long long react) {
  k_dg_arm<<<1, 32, 0, st>>>(S.ctl, steps, rebuild, react);
}

void launch_dg_next(const Sys& S, cudaStream_t st, unsigned int theta) {
  k_dg_next<<<1, 32, 0, st>>>(S.ctl, S.has_rx, theta);
}

}  // namespace prx
