// Level-set step buffers and launch entry points.
#pragma once
#include <functional>

#include "common.cuh"

namespace etd {

struct LevelsetBufs {
  uint8_t* lflag;   // per list entry: tube / validity bits
  uint32_t* bits;   // bit planes of the work-set build (one bit per node)
  int* list;        // grid indices of the work set, grid order
  ushort4* lcoord;  // per list entry: the node's axis indices
  int* slist;       // RK stage list: work-list positions of the update set
  int* count;       // [0] list length, [1] [2] stage-list front / back counts
  int* cta_count;   // per-CTA counts for the in-kernel compaction
  int* sw;          // extension sweep list: [1..3] entries per level, [5..7] placement cursors
  double* vmax;     // [0] max Stefan speed on the tube
  int* nsub;        // [0] advection substeps of the last call
  int* info;        // last call: list and tube sizes, substeps (see levelset_last_stats)
  double* nrm;      // N x list capacity: unit normals (compact)
  double* V;        // list capacity: Stefan speed (compact)
  double* S0;       // list capacity: sign function of reinitialisation (compact)
  double* q[6];     // grid: extension ping-pong buffers (u_nn, u_n, u)
  double* p1;       // grid: RK stage values
  double* p2;
  int* gidx;        // grid: work-list position of each work-set node (valid where list[gidx[p]] == p)
};

LevelsetBufs levelset_carve(const GridDev& g, const std::function<char*(size_t)>& take);

// mixed: FP32 WENO/Godunov arithmetic except for the reinitialisation within
// h of the interface, FP32 extension sweeps and FP32 Stefan-speed
// interpolation (FP64 everywhere when false)
cudaError_t launch_levelset_advance(const GridDev& g, const LevelsetBufs& b, DevStatus* st, const uint8_t* kind,
                                    double* phi, double* u, double dt, double mu, bool reinit, bool mixed,
                                    cudaStream_t stream);
cudaError_t launch_levelset_prepare(const GridDev& g, const LevelsetBufs& b, DevStatus* st, double* phi, bool reinit,
                                    bool mixed, cudaStream_t stream);

}  // namespace etd
