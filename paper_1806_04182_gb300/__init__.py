"""GB300-native method-of-lines substep of arXiv:1806.04182 (wave, MHD, CCZ4)."""
