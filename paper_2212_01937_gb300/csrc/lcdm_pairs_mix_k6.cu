// Pair-kernel instantiations: precision mix, 6 tangent directions.
#include "lcdm_launch.cuh"
namespace lcdm {
LCDM_DEFINE_TABLE(table_mix_k6, 1, 6)
}
