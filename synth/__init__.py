"""Seeded synthetic workloads for the epoch-model tree likelihood.

This module is the one thing the CPU oracle (``oracle/``) and the CUDA
library (``paper_1309_3075_b300``) both consume.  It holds none of the
likelihood's arithmetic: it draws trees, model parameters and data, writes
the *raw* rate matrices Q_s (and dQ_s/dtheta) from their textbook
definitions (HKY85, GTR, Goldman-Yang 1994, asymmetric discrete-trait CTMC),
draws discrete-gamma category rates with scipy, and simulates alignments by
exact jump-chain (Gillespie) simulation of the CTMC path, switching Q at the
epoch boundaries.  It never forms a transition matrix, a product of
transition matrices or a partial likelihood.  Both sides normalise Q_s and
do everything else themselves.

The shapes follow the paper's workloads (HKY with kappa 1..10, GY94 with
omega 0.1..1, 2..4 epochs, 7..61 states, 100..1000 taxa); the paper's
empirical data sets are not used.
"""
from synth.workloads import (  # noqa: F401
    Workload,
    BatchWorkload,
    coalescent_tree,
    discrete_gamma,
    hky_raw,
    gtr_raw,
    gy94_raw,
    asym_raw,
    simulate_alignment,
    compress_patterns,
    hky_8taxa,
    gtr_500taxa,
    gy94_128taxa,
    asym50_forest,
    small_nucleotide,
    small_codon,
    tiny_tree_workload,
    exchange_raw,
    flu_seasonal,
    amino_acid,
    GENETIC_CODE,
    SENSE_CODONS,
)
