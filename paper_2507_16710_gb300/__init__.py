"""GB300-native single-device sort (sm_103a) behind a C ABI.

The rank-local sort of the paper's distributed sample sort (Sec. IV-A), with
the sort / sortperm / by-key operations of its building blocks (Sec. II-B), in
Julia isless order.  Python here only marshals arguments: the compiled library
``lib/libak_sort.so`` (built by ``_build.build()``) does all the work.
"""
from ._lib import (  # noqa: F401
    AK_ASCENDING, AK_BF16, AK_DESCENDING, AK_F16, AK_F32, AK_F64, AK_I16, AK_I32, AK_I64, AK_I128, AK_U128,
    AK_OP_SORT,
    AK_OP_SORT_PAIRS, AK_OP_SORT_SEGMENTED, AK_OP_SORTPERM, AK_OP_SORTPERM_LOWMEM, AK_PATH_AUTO, AK_PATH_BLOCK,
    AK_PATH_LEARNED, AK_PATH_MERGE, AK_PATH_RADIX, AK_TILE_CONFIGS, AK_U16, AK_U32, AK_U64, EXPORTED, LIB_PATH,
    AK_DEBUG_SKIP_FIRST_TILE, AK_DEBUG_NO_PREFETCH, AK_DEBUG_NO_PACK, AK_MAX_PASSES,
    AkError, Info, Options, ak_autotune, ak_autotune_segmented, autotune_temp_bytes, ak_autotune_clear, ak_autotune_load, ak_autotune_save,
    ak_last_info, ak_learned_knots, ak_learned_loss_grad, ak_sort, ak_sort_pairs,
    ak_sort_segmented, ak_sort_static_scratch, ak_sort_temp_bytes, ak_sortperm, ak_sortperm_lowmem, ak_status_check, ak_status_string,
    ak_accumulate, accumulate_temp_bytes, ak_searchsortedfirst, ak_searchsortedlast, ak_segment_capacity, ak_version, dtype_code, key_code, load, order_code, temp_bytes, workspace,
)
