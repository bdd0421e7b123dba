"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package only draws random numbers and builds planted data models. It holds
none of the gamma-EigenGame arithmetic: no mat-vec, no update rule, no
eigensolver. Both the CPU oracle and the CUDA path receive their inputs from
here, so neither depends on the other.
"""
from .planted import (  # noqa: F401
    PlantedCCA, PlantedLowRankCCA, planted_cca, planted_lowrank_cca, planted_pca,
    draw_rows, draw_pca_rows, draw_lda_rows, planted_lda, random_unit_columns, quantize_e4m3_rows,
    finite_dataset_indices, config_c1, config_c2, config_c3, config_c4, config_c5,
    planted_ica, draw_ica_rows, ICA_KURTOSIS,
)
