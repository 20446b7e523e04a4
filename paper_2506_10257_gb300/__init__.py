"""GB300-native robust PCA (principal component pursuit) for ultrasound frame windows."""
