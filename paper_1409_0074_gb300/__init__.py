"""GB300-native local approximate GP prediction (Gramacy & Haaland, arXiv:1409.0074)."""
