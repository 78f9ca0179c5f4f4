"""GB300-native exact planted motif search (PMS8 hot path, Nicolae & Rajasekaran).

Importing the package is cheap: the CUDA library is loaded on first use by
`paper_1307_0571_gb300.pms`, which fails loudly when the compiled library is missing.
"""
