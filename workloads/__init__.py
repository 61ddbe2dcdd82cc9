"""Seeded synthetic workloads and index-construction helpers.

This package only builds INPUTS: base vectors, queries, the IVF-PQ index arrays
(centroids, codebooks, codes, list assignment) and exact ground truth for
recall. It holds none of the search arithmetic that is checked (coarse
distances, LUT construction, quantisation, ADC scan, top-k, precision choice);
both the CPU oracle and the CUDA library take its arrays as given.
"""
from .synth import CONFIGS, make_dataset, make_queries, zipf_nprobe, mixed_k  # noqa: F401
from .index_train import train_ivfpq  # noqa: F401
from .groundtruth import exact_knn, recall_at  # noqa: F401
