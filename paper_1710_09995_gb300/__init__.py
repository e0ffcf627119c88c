"""GB300-native structured-grid finite-volume hot path (arXiv 1710.09995, Sec. 2).

Importing the package loads nothing native; `paper_1710_09995_gb300.gbcfd` loads the CUDA
library (and raises if it is missing), `paper_1710_09995_gb300.cases` holds the seeded inputs.
"""
