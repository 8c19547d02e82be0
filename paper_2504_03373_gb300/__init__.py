"""GB300-native GSVD-MUSIC sound source localization (arXiv 2504.03373)."""
