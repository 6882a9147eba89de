"""GB300-native Shannon / Tsallis mutual information for 3D registration."""
