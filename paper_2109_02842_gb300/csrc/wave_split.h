// Host arithmetic of the tensor-core back-projection's split into its full
// waves and its last partial wave, and of the pixels the full waves finish
// (no CUDA: the CPU tests compile it with a plain C++ compiler).
#pragma once

#include <algorithm>

struct WaveSplit {
    int full;   // blocks of the full waves (0: no split)
    int cols;   // image pixels (y-major, x fastest) whose every channel part
                // is in the full waves: [0, cols)
};

// total: blocks of one back-projection with one bin block; wave: blocks
// resident at once; nsplit: channel parts per tile; nbx: tiles along x;
// tile_y: pixel rows per tile; nx, ny: the image grid. Blocks are ordered
// (tile x, tile y, part), x fastest, so tile t's last part is block
// (nsplit - 1) T + t with T = total / nsplit tiles, and the tiles finished
// by the first `full` blocks are a prefix; the pixels of their whole rows of
// tiles are a prefix of the image plane. A split is made only when the full
// waves leave a partial last wave and finish at least one row of tiles.
inline WaveSplit bp_wave_split(int total, int wave, int nsplit, int nbx, int tile_y, int nx,
                               int ny) {
    WaveSplit r{0, 0};
    if (total <= 0 || wave <= 0 || nsplit <= 0 || nbx <= 0 || tile_y <= 0) return r;
    const int full = total / wave * wave;
    const int T = total / nsplit;
    const int tiles_done = std::max(0, full - (nsplit - 1) * T);
    const int rows = std::min(ny, tiles_done / nbx * tile_y);
    if (full > 0 && full < total && rows > 0) {
        r.full = full;
        r.cols = rows * nx;
    }
    return r;
}
