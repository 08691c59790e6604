// Tensor-core (tcgen05) numeric phase: declarations shared with the driver.
#pragma once

#include "rdm_internal.cuh"

namespace rdm {

// Test settings of the tensor-core path (rdm_set_test_knobs); zeros keep the
// production behaviour.
struct TcKnobs {
    long long wait_cycles = 0;  // bound of every mbarrier wait in SM clock cycles (0: ~2 s)
    int hold = 0;               // 1: the MMA thread first waits for a flag that nothing sets
    int window_words = 0;       // bitmap window of the tile-plan builders in 32-column words
                                // (0: 512, i.e. 16,384 columns; wider windows take the serial merge)
    int block_copies = 0;       // 1: planes at their own positions and one bulk copy per block
};

// work buffers of the tensor-core path (tile lists, per-tile K-step lists)
struct TcWork {
    TcKnobs knobs;
    DevBuf<uint16_t> zero;      // zero operand blocks: one per CTA and K-step slot
    DevBuf<int> tiles;          // per tile: job, I, -, nsteps, mask slot[TBM x TBN], column j[TBN]
    DevBuf<int> tile_cnt, tile_off;
    DevBuf<int> step_cnt;
    DevBuf<int64_t> step_off;
    DevBuf<int> steps;          // per K-step: TBM A block indices, TBN B block indices (-1 = zero)
    DevBuf<int> counters;       // [0]: error bits of the product kernel
    DevBuf<int> scan32;
    DevBuf<int64_t> scan64;
    DevBuf<float> scale;        // per matrix: power-of-two scale of its operand planes
    DevBuf<unsigned> mx;        // per matrix: largest block norm (bit pattern)
    DevBuf<int> mat_first;      // per matrix: first global block index (nmat+1)
    DevBuf<int> tpos;           // per block (i, k) of the input set: global index of block (k, i)
    DevBuf<int> pre_err;        // error bits of the operand preparation (8: a transposed block missing)
    bool tpos_valid = false;    // the planes sit at tpos and the K-step lists point there
};

// work buffers of the slice-product (FP64-class) tensor-core path
struct OzWork {
    DevBuf<int> e;              // per global row of matrix 0: exponent e_r of its scale 2^e_r
    DevBuf<int> row_of;         // block row of every block of matrix 0
    DevBuf<uint16_t> slices;    // 7 bf16 slices per element of matrix 0 (14 KB per 32 x 32 block)
    DevBuf<uint16_t> zero;      // zero blocks: one per CTA and K-step slot
};

struct TcPlan {
    int ntile;
    int64_t nsteps;
};

// Block sizes the tensor-core kernel handles (16, 32, 64), and the block rows
// of its 128 x 256 tiles for block size b (128 / b; 4 for other sizes, the
// super-row of the CUDA-core path).
bool tc_block_size_ok(int b);
int tc_tile_rows(int b);

// Convert the FP64 master values of `in` into hi/lo operand planes of
// arithmetic `ar` in the K-major core-matrix layout of the MMA.  For fp16
// every matrix is first scaled by a power of two (from its largest block
// norm) so that its values sit in the normal range of fp16; the product
// kernel divides the scale back out per job.
void prepare_operands(MatSet &in, Arith ar, TcWork &w, cudaStream_t st);

// Tile lists of one multiplication step from the output mask, for the jobs
// selected by job_mask (per system tier) and the super-row units
// [unit0, unit1) (unit = job * ceil(NB/TR) + I covers block rows
// TR I .. TR I + TR - 1 of the job, TR = tc_tile_rows(b)).
TcPlan build_tc_plan(const MatSet &in, const JobTable &jt, const SysDev &sd, const int *out_rp,
                     const int *mcol, TcWork &w, JobMask job_mask, int unit0, int unit1, cudaStream_t st);

// Numeric phase on the tensor cores; same output contract as
// launch_numeric_simt for the slots of active systems.  Returns the flops
// issued to the tensor cores.
double launch_numeric_tc(const NumArgs &a, const MatSet &in, const JobTable &jt, Arith ar, TcWork &w,
                         int NB, const TcPlan &plan, cudaStream_t st);

// FP64-class products X0^2 on the tensor cores from exact bf16 slices
// (32 x 32 blocks; k_oz.cu): the slices and row scales of matrix 0 of `in`,
// the tile lists (128 x 64 tiles, job 0 only), and the launch (same output
// contract as the other numeric launches; returns the MMA flops issued).
void prepare_oz_operands(const MatSet &in, OzWork &w, cudaStream_t st);
TcPlan build_oz_plan(const MatSet &in, const JobTable &jt, const SysDev &sd, const int *out_rp, const int *mcol,
                     TcWork &w, JobMask job_mask, int unit0, int unit1, cudaStream_t st);
double launch_numeric_oz(const NumArgs &a, const MatSet &in, const int *mcol, OzWork &ow, TcWork &w,
                         const TcPlan &plan, cudaStream_t st);

}  // namespace rdm
