// Pair-kernel instantiations: precision mix, 0 tangent directions.
#include "lcdm_launch.cuh"
namespace lcdm {
LCDM_DEFINE_TABLE(table_mix_k0, 1, 0)
}
