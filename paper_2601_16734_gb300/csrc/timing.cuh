// Optional per-phase timing with CUDA events on the context's stream.
// When enabled (seemps_set_timing), every phase records a start/end event
// pair; seemps_get_timing() (or a full event pool) synchronises the stream
// and accumulates the elapsed milliseconds per phase.
#pragma once

#include "common.cuh"

int timing_begin(seemps_ctx* ctx, int phase);  // returns a slot, or -1 when timing is off
void timing_end(seemps_ctx* ctx, int slot);
seemps_status timing_flush(seemps_ctx* ctx);

struct PhaseTimer {
  seemps_ctx* ctx;
  int slot;
  PhaseTimer(seemps_ctx* c, int phase) : ctx(c), slot(timing_begin(c, phase)) {}
  ~PhaseTimer() { timing_end(ctx, slot); }
};
