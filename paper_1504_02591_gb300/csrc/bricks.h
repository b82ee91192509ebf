// bricks.h: brick-sorted particle pipeline (pack, counting sort, binned deposit, sorted gather).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace rg {

constexpr int kBrick = 8;                         // cells per brick edge
constexpr int kBrickHalo = kBrick + 1;            // CIC touches one node beyond the brick
constexpr int kBrickNodes = kBrickHalo * kBrickHalo * kBrickHalo;   // 729
constexpr long long kSortChunk = 1LL << 25;       // particles sorted together (meshes >= 256)
constexpr long long kSortChunkSmall = 1LL << 22;  // ... on smaller meshes
inline long long sort_chunk(int n) { return n >= 256 ? kSortChunk : kSortChunkSmall; }
constexpr int kFracBits = 21;                     // fixed-point fraction of a cell per axis

struct BrickBuffers {
  int n;                 // mesh side (multiple of 8)
  int nb;                // bricks per axis
  double scale;          // n / L
  long long chunk;       // particles per sort (sort_chunk(n))
  uint32_t* hist;        // nb^3 counts
  uint32_t* offs;        // nb^3 + 1 exclusive offsets
  uint32_t* bsum;        // scan block sums (<= 4096)
  uint4* rec;            // kSortChunk sorted records: packed x, y, z (cell << 21 | frac), weight bits
  uint32_t* perm;        // kSortChunk: sorted slot -> index within the chunk
  uint32_t* key;         // kSortChunk: brick of each particle (input order)
  uint32_t* rank;        // kSortChunk: arrival rank of each particle within its brick
  uint4* pre;            // kSortChunk: packed records in input order (count -> scatter); free after
                         // the scatter (a retained sort's shift writes its float32 shifts here)
};

size_t brick_scratch_bytes(int n);
// carve the brick buffers out of a workspace region of brick_scratch_bytes(n)
BrickBuffers brick_buffers(char* base, int n, double L);

// count -> scan -> scatter of particles [0, np) (np <= kSortChunk)
cudaError_t brick_sort(const BrickBuffers& b, const void* pos, int dtype, const float* w, long long np,
                       cudaStream_t st);

// CIC deposit of the sorted chunk into rho (shared-memory brick tiles, then global atomics);
// per-block weight sums into partials[0 .. brick_grid())
cudaError_t brick_deposit(const BrickBuffers& b, float* rho, double* partials, cudaStream_t st);
int brick_grid();

struct BrickShiftArgs {
  const float* psi[3];   // real Psi components
  const float* off;      // 3 N node offsets from the observer (radial LOS)
  double H;              // cell size
  int is_galaxy;
  float f;
  int los_mode;
  float3 los;
  int periodic;
  double L;
  const void* pos;       // original positions of the chunk (pos_out only)
  int dtype;
  float* shift;          // chunk outputs, original order
  double* pos_out;       // or null
};

// CIC interpolation of Psi and the shift for the sorted chunk (one warp per brick)
cudaError_t brick_shift(const BrickBuffers& b, const BrickShiftArgs& a, cudaStream_t st);

}  // namespace rg
