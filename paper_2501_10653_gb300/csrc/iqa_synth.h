// iqa_synth.h -- device-side synthetic sky epochs (serving loop input
// generation; see iqa_synth.cu for the exact recipe).
#pragma once

#include <cuda_runtime.h>

namespace iqa {

constexpr int kSynthBin = 64;     // pixels per side of a catalogue bin and of
                                  // a generator work unit
constexpr int kSynthMaxDrop = 8;  // sources a request may drop

// A reference catalogue in device memory.
struct SynthCatalog {
    int nsrc;
    int N;
    int bins_per_row;            // N / kSynthBin (rounded up)
    float noise_sigma;
    const int *x;                // integer source centres
    const int *y;
    const float *flux;           // peak flux
    const int *half;             // profile half-width h (window 2h+1)
    const int *profile_off;      // start of source i's profile in `profile`
    const float *profile;        // concatenated 1-D profiles
    const int *bin_start;        // CSR over bins: sources whose window meets bin
    const int *bin_src;          // source indices, catalogue order
};

// One epoch to render.
struct SynthJob {
    const SynthCatalog *cat;     // device pointer
    void *out;                   // N*N storage elements
    long long blocks_begin;      // first catalogue bin (work unit) of this job
    unsigned long long seed;
    int N;
    int ndrop;
    int drop[kSynthMaxDrop];     // catalogue indices left out of this epoch
    int add_src;                 // -1, or a source whose profile a transient uses
    int add_x, add_y;            // transient centre
    float add_flux;              // transient peak flux
};

// Resident generator blocks per SM; a grid of num_sms * kSynthBlocksPerSM
// keeps every SM full (the kernel loops over the bins).
constexpr int kSynthBlocksPerSM = 8;

// Renders every job of the table (at most 64); header = {njobs, total_bins}
// in device memory (so a captured graph can replay it with new contents).
// N must be a multiple of kSynthBin (at most 2^20), and a bin may list at most
// 64 sources.
cudaError_t launch_synth(int dtype, const SynthJob *jobs, const long long *header, int grid,
                         cudaStream_t st);

}  // namespace iqa
