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

__global__ void k_dgb_arm(BatchCtl* c, unsigned long long steps, unsigned long long phase,
                          unsigned long long theta, int any_rx, unsigned long long rebuild,
                          unsigned long long react) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    c->steps_left = steps;
    c->phase = phase;
    c->theta = theta;
    c->any_rx = any_rx;
    c->dg_rebuild = rebuild;
    c->dg_react = react;
  }
}

// After a batch step (the last member's epilogue left its decision in
// rebuild_now): the rebuild of the members that need one, the reaction step
// when the batch's phase wraps, the next step.
__global__ void k_dgb_next(BatchCtl* c) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  bool ok = true;
  if (c->rebuild_now)
    ok = cudaGraphLaunch((cudaGraphExec_t)c->dg_rebuild, cudaStreamGraphTailLaunch) == cudaSuccess;
  c->phase = c->theta ? (c->phase + 1ull) % c->theta : 0ull;
  if (ok && c->any_rx && c->phase == 0ull)
    ok = cudaGraphLaunch((cudaGraphExec_t)c->dg_react, cudaStreamGraphTailLaunch) == cudaSuccess;
  if (ok && c->steps_left > 1ull) {
    c->steps_left -= 1ull;
    ok = cudaGraphLaunch(cudaGetCurrentGraphExec(), cudaStreamGraphTailLaunch) == cudaSuccess;
  } else {
    c->steps_left = 0ull;
  }
  if (!ok) c->dg_err = 1;
}

}  // namespace

void launch_dgb_arm(BatchCtl* c, cudaStream_t st, unsigned long long steps, unsigned long long phase,
                    unsigned long long theta, int any_rx, unsigned long long rebuild,
                    unsigned long long react) {
  k_dgb_arm<<<1, 32, 0, st>>>(c, steps, phase, theta, any_rx, rebuild, react);
}

void launch_dgb_next(BatchCtl* c, cudaStream_t st) { k_dgb_next<<<1, 32, 0, st>>>(c); }

void launch_dg_arm(const Sys& S, cudaStream_t st, unsigned long long steps,
                   unsigned long long rebuild, unsigned long long react) {
  k_dg_arm<<<1, 32, 0, st>>>(S.ctl, steps, rebuild, react);
}

void launch_dg_next(const Sys& S, cudaStream_t st, unsigned int theta) {
  k_dg_next<<<1, 32, 0, st>>>(S.ctl, S.has_rx, theta);
}

}  // namespace prx
