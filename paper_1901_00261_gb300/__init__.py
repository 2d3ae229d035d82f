"""GB300-native compact 6th/8th-order gas-kinetic scheme (arXiv:1901.00261)."""
