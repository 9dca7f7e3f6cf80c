"""GB300-native MMH-MH privacy amplification (arXiv 2105.13678)."""
