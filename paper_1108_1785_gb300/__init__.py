"""GB300-native flow-record analysis: the data-parallel hot path of G-NetMon (per-site
transfer rates of NetFlow records by longest-prefix match), as CUDA kernels for sm_103a
behind a C ABI (include/gnm.h). ``gnm`` is the Python binding; ``build`` compiles the
library in-tree."""
from . import build  # noqa: F401
from .gnm import (Context, GnmError, Plan, Records, Stream, lib, NO_SITE, LOOKUP_AUTO, LOOKUP_BSEARCH,  # noqa: F401
                  LOOKUP_RMI, LOOKUP_RADIX, LOOKUP_HASH24, PLACE_AUTO, PLACE_SMEM, PLACE_L2, PLACE_STAGED, AGG_AUTO, AGG_DIRECT, AGG_WARP,
                  ADMIN_OR, ADMIN_AND, ROOT_LINEAR, ROOT_MLP, TABLE_AUTO, TABLE_DIRECT, TABLE_HASH,
                  TABLE_GLOBAL, TABLE_PARTITION, SPLIT_AUTO, SPLIT_FUSED, SPLIT_TWO_KERNELS, registry_flatten)
