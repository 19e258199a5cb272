"""GB300-native contrast-maximisation loss + gradient (arXiv 2412.06359)."""
