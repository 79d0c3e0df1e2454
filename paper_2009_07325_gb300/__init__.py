"""GB300-native IMM (RR-set sampling + greedy max coverage)."""
