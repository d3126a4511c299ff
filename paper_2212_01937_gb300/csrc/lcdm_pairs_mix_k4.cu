// Pair-kernel instantiations: precision mix, 4 tangent directions.
#include "lcdm_launch.cuh"
namespace lcdm {
LCDM_DEFINE_TABLE(table_mix_k4, 1, 4)
}
