"""GB300-native dense generalized Hermitian eigensolver (H C = S C Lambda, Eq. 2)."""
