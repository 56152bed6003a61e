"""Seeded synthetic snapshot matrices.

This package only draws inputs.  It holds none of the method's arithmetic,
so both the FP64 oracle and the GPU path may import it.
"""
from .fields import (  # noqa: F401
    GridSpec, heat_field, blob_field, spiked_blob_field, tanh_front_field, low_rank_matrix,
    pivot_gap_matrix, to_bf16_bits, bf16_bits_to_f64, make_workload, WORKLOADS,
    BatchSpec, batch_specs, make_batch_matrix,
    LEARNED_FIELDS, learned_specs, learned_heldout_specs, learned_matrix, learned_spec_from_meta,
)
