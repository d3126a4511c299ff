// Pair-kernel instantiations: precision mix, 3 tangent directions.
#include "lcdm_launch.cuh"
namespace lcdm {
LCDM_DEFINE_TABLE(table_mix_k3, 1, 3)
}
